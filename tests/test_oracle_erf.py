"""Pins for the oracle's Erf maps (the activation erf(x), one of the
activations of the paper's Myrtle architecture search).

* erf_map against a 1-D adaptive quadrature built on a different identity:
  E_z[erf(a + b z)] = erf(a / sqrt(1 + 2 b^2)) for z ~ N(0, 1), integrated
  over the remaining Gaussian variable; and against a plain 2-D
  Gauss-Hermite rule of 160^2 nodes (the integrand is smooth, so the rule
  converges fast: at q = 4 the error falls from 1.6e-8 at 80 nodes to 2e-16).
* erf_derivative_map (E[erf' erf'], the NTK's derivative kernel) against the
  2-D Gauss-Hermite rule.
* Special values: zero at K = 0, odd in K, the c = 1 limit equal to
  E[erf(u)^2] by 1-D quadrature.
* Monte Carlo: finite random networks with erf activations and one hidden
  layer (pre-activations exactly Gaussian at any width) -- the readout
  covariance (NNGP) and the empirical NTK (gradients by autograd, NTK
  parameterisation) -- within sampling error of the oracle's Myrtle
  recursion with act = "erf".
"""

import math

import numpy as np
import pytest
import torch
from scipy import integrate, special, stats

from nkdata import SEED_MC
from oracle import Arch, erf_derivative_map, erf_map, myrtle_block, myrtle_ntk_block

F64 = torch.float64
QS = [(1.0, 1.0), (0.3, 2.5), (4.0, 0.07)]
CS = [-1.0, -0.9, -0.4, 0.0, 0.25, 0.7, 0.99, 1.0]


def _t(v):
    return torch.tensor(v, dtype=F64)


def expect_erf_product(q1, q2, c):
    """E[erf(u) erf(v)], u = sqrt(q1) z1, v = sqrt(q2)(c z1 + s z2), s = sqrt(1 - c^2):
    the inner expectation over z2 is erf(sqrt(q2) c z1 / sqrt(1 + 2 q2 s^2))."""
    s2 = max(0.0, 1.0 - c * c)

    def inner(z1):
        return special.erf(math.sqrt(q1) * z1) * special.erf(math.sqrt(q2) * c * z1 / math.sqrt(1.0 + 2.0 * q2 * s2)) \
            * stats.norm.pdf(z1)

    val, _ = integrate.quad(inner, -np.inf, np.inf, epsabs=1e-14, epsrel=1e-13, limit=200)
    return val


def _gauss_hermite_2d(fn, q1, q2, c, n=160):
    x, w = np.polynomial.hermite_e.hermegauss(n)
    w = w / w.sum()
    Z1, Z2 = np.meshgrid(x, x, indexing="ij")
    u = math.sqrt(q1) * Z1
    v = math.sqrt(q2) * (c * Z1 + math.sqrt(max(0.0, 1.0 - c * c)) * Z2)
    return float((np.outer(w, w) * fn(u) * fn(v)).sum())


@pytest.mark.parametrize("q1,q2", QS)
def test_erf_map_matches_quadrature(q1, q2):
    for c in CS:
        K = c * math.sqrt(q1 * q2)
        got = float(erf_map(_t(K), _t(q1), _t(q2)))
        want = expect_erf_product(q1, q2, c)
        assert abs(got - want) <= 1e-11, (q1, q2, c, got, want)


@pytest.mark.parametrize("q1,q2", QS)
def test_erf_maps_match_gauss_hermite(q1, q2):
    derf = lambda z: 2.0 / math.sqrt(math.pi) * np.exp(-z * z)  # noqa: E731
    for c in [-0.8, 0.0, 0.4, 0.9]:
        K = c * math.sqrt(q1 * q2)
        got = float(erf_map(_t(K), _t(q1), _t(q2)))
        assert abs(got - _gauss_hermite_2d(special.erf, q1, q2, c)) <= 1e-10, (q1, q2, c)
        gotd = float(erf_derivative_map(_t(K), _t(q1), _t(q2)))
        assert abs(gotd - _gauss_hermite_2d(derf, q1, q2, c)) <= 1e-10 * max(1.0, gotd), (q1, q2, c)


def test_erf_map_special_values():
    q1, q2 = _t(0.7), _t(1.9)
    assert float(erf_map(_t(0.0), q1, q2)) == 0.0
    for K in [0.1, 0.5, 1.1]:
        assert float(erf_map(_t(-K), q1, q2)) == pytest.approx(-float(erf_map(_t(K), q1, q2)), abs=1e-15)
    # c = 1, q1 = q2 = q: E[erf(u)^2] for u ~ N(0, q)
    for q in [0.05, 1.0, 6.0]:
        want, _ = integrate.quad(lambda z: special.erf(math.sqrt(q) * z) ** 2 * stats.norm.pdf(z), -np.inf, np.inf,
                                 epsabs=1e-14, epsrel=1e-13)
        assert float(erf_map(_t(q), _t(q), _t(q))) == pytest.approx(want, abs=1e-12)


@pytest.fixture(scope="module")
def tiny():
    rng = np.random.default_rng(SEED_MC + 3)
    return torch.tensor(rng.standard_normal((3, 4, 4, 2)))


def _nngp_draws(sw2, sb2, X, width, draws, gen):
    """Readout covariances [draws, B, B] of one-hidden-layer erf networks (the
    readout expectation taken exactly given the hidden layer)."""
    B, H, W, C = X.shape
    x0 = X.permute(0, 3, 1, 2)
    out = []
    for _ in range(draws):
        w = torch.randn(width, C, 3, 3, dtype=F64, generator=gen) * math.sqrt(sw2 / (C * 9))
        b = torch.randn(width, dtype=F64, generator=gen) * math.sqrt(sb2)
        h = torch.erf(torch.nn.functional.conv2d(x0, w, b, padding=1))
        g = h.mean(dim=(2, 3))  # [B, width]
        out.append(sw2 / width * g @ g.T + sb2)
    return torch.stack(out)


def test_erf_nngp_monte_carlo_one_hidden_layer(tiny):
    sw2, sb2 = 2.0, 0.1
    want = myrtle_block(Arch((1,), act="erf"), sw2, sb2, tiny, tiny)
    gen = torch.Generator().manual_seed(SEED_MC + 11)
    covs = _nngp_draws(sw2, sb2, tiny, width=2048, draws=64, gen=gen)
    mean = covs.mean(0)
    se = covs.std(0) / math.sqrt(covs.shape[0])
    assert float(((mean - want).abs() / se).max()) < 4.5, (mean, want, se)
    assert float(((mean - want).abs() / want.abs()).max()) < 0.01


def _empirical_ntk_erf(sw2, sb2, X, width, gen):
    B, H, W, C = X.shape
    w = torch.randn(width, C, 3, 3, dtype=F64, generator=gen).requires_grad_()
    b = torch.randn(width, dtype=F64, generator=gen).requires_grad_()
    wo = torch.randn(width, dtype=F64, generator=gen).requires_grad_()
    bo = torch.randn((), dtype=F64, generator=gen).requires_grad_()
    params = [w, b, wo, bo]

    def f(x):
        h = torch.nn.functional.conv2d(x.permute(2, 0, 1)[None], w * math.sqrt(sw2 / (C * 9)), b * math.sqrt(sb2),
                                       padding=1)
        g = torch.erf(h).mean(dim=(2, 3))[0]
        return (wo * g).sum() * math.sqrt(sw2 / width) + bo * math.sqrt(sb2)

    G = torch.stack([torch.cat([gr.reshape(-1) for gr in torch.autograd.grad(f(X[a]), params)])
                     for a in range(B)])
    return G @ G.T


def test_erf_ntk_monte_carlo_one_hidden_layer(tiny):
    sw2, sb2 = 2.0, 0.1
    _, want = myrtle_ntk_block(Arch((1,), act="erf"), sw2, sb2, tiny, tiny)
    gen = torch.Generator().manual_seed(SEED_MC + 12)
    draws = torch.stack([_empirical_ntk_erf(sw2, sb2, tiny, 512, gen) for _ in range(96)])
    mean = draws.mean(0)
    se = draws.std(0) / math.sqrt(draws.shape[0])
    assert float(((mean - want).abs() / se).max()) < 4.5, (mean, want, se)
    assert float(((mean - want).abs() / want.abs()).max()) < 0.02


def test_erf_myrtle_symmetric_psd(tiny):
    K = myrtle_block(Arch((2, 1, 0), act="erf"), 2.0, 0.01, tiny, tiny)
    assert torch.allclose(K, K.T, rtol=1e-13)
    assert float(torch.linalg.eigvalsh(K).min()) >= -1e-13 * float(K.abs().max())
