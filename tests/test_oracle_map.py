"""Pins for the oracle's ReLU arc-cosine map (stax.Relu, Appendix A listings).

The closed form is checked against an independent numerical expectation:
E[relu(u) relu(v)] for centred Gaussian (u, v) computed by integrating the
textbook rectified-Gaussian mean E_z[relu(a + s z)] = a Phi(a/s) + s phi(a/s)
over the remaining variable with adaptive quadrature, and against a plain 2-D
Gauss-Hermite rule.  Special values and the derivative are pinned too.
"""

import math

import numpy as np
import pytest
import torch
from scipy import integrate, stats

from oracle import relu_map

F64 = torch.float64


def expect_relu_product(q1, q2, c):
    """E[relu(u) relu(v)], u = sqrt(q1) z1, v = sqrt(q2)(c z1 + s z2)."""
    s = math.sqrt(max(0.0, 1.0 - c * c))

    def inner(z1):
        a = c * z1
        if s == 0.0:
            m = max(a, 0.0)
        else:
            m = a * stats.norm.cdf(a / s) + s * stats.norm.pdf(a / s)
        return z1 * m * stats.norm.pdf(z1)

    val, err = integrate.quad(inner, 0.0, np.inf, epsabs=1e-14, epsrel=1e-13, limit=200)
    return math.sqrt(q1 * q2) * val


CS = [-1.0, -1.0 + 1e-12, -0.9, -0.5, -0.1, 0.0, 0.3, 0.7071, 0.95, 1.0 - 1e-12, 1.0]
QS = [(1.0, 1.0), (0.3, 2.5), (4.0, 0.07)]


@pytest.mark.parametrize("q1,q2", QS)
def test_map_matches_quadrature(q1, q2):
    for c in CS:
        K = c * math.sqrt(q1 * q2)
        got = float(relu_map(torch.tensor(K, dtype=F64), torch.tensor(q1, dtype=F64),
                             torch.tensor(q2, dtype=F64)))
        want = expect_relu_product(q1, q2, c)
        assert abs(got - want) <= 1e-11 * math.sqrt(q1 * q2), (q1, q2, c, got, want)


def test_map_matches_gauss_hermite_2d():
    # plain 2-D Gauss-Hermite (probabilists'), 96^2 nodes; the kink of relu
    # limits its accuracy, so this is a coarse second opinion
    x, w = np.polynomial.hermite_e.hermegauss(96)
    w = w / w.sum()
    Z1, Z2 = np.meshgrid(x, x, indexing="ij")
    W2 = np.outer(w, w)
    for q1, q2 in QS:
        for c in [-0.8, 0.0, 0.4, 0.9]:
            s = math.sqrt(1 - c * c)
            u = math.sqrt(q1) * Z1
            v = math.sqrt(q2) * (c * Z1 + s * Z2)
            gh = float((W2 * np.maximum(u, 0) * np.maximum(v, 0)).sum())
            got = float(relu_map(torch.tensor(c * math.sqrt(q1 * q2), dtype=F64),
                                 torch.tensor(q1, dtype=F64), torch.tensor(q2, dtype=F64)))
            assert abs(got - gh) <= 2e-3 * math.sqrt(q1 * q2)


def test_map_special_values():
    q = torch.tensor(1.7, dtype=F64)
    qp = torch.tensor(0.4, dtype=F64)
    # c = 1 with q = q': E[relu(u)^2] = q / 2
    assert abs(float(relu_map(q, q, q)) - 0.85) < 1e-15
    # c = -1: relu(u) relu(-u) = 0
    assert abs(float(relu_map(-torch.sqrt(q * qp), q, qp))) < 1e-15
    # c = 0: independent, E[relu]^2 = q/(2 pi) -> sqrt(q q')/(2 pi)
    assert abs(float(relu_map(torch.tensor(0.0, dtype=F64), q, qp))
               - math.sqrt(1.7 * 0.4) / (2 * math.pi)) < 1e-15
    # zero variance gives zero
    assert float(relu_map(torch.tensor(0.0, dtype=F64), torch.tensor(0.0, dtype=F64), q)) == 0.0


def test_map_derivatives_by_central_differences():
    # dKt/dK = (pi - theta)/(2 pi); dKt/dq = (Kt - K (pi - theta)/(2 pi)) / (2 q)
    h = 1e-6
    for q1, q2 in QS:
        for c in [-0.9, -0.2, 0.0, 0.5, 0.99]:
            K = torch.tensor(c * math.sqrt(q1 * q2), dtype=F64, requires_grad=True)
            a = torch.tensor(q1, dtype=F64, requires_grad=True)
            b = torch.tensor(q2, dtype=F64, requires_grad=True)
            out = relu_map(K, a, b)
            out.backward()
            f = lambda k, x, y: float(relu_map(torch.tensor(k, dtype=F64), torch.tensor(x, dtype=F64),
                                               torch.tensor(y, dtype=F64)))
            k0 = float(K.detach())
            dK = (f(k0 + h, q1, q2) - f(k0 - h, q1, q2)) / (2 * h)
            dq1 = (f(k0, q1 + h, q2) - f(k0, q1 - h, q2)) / (2 * h)
            dq2 = (f(k0, q1, q2 + h) - f(k0, q1, q2 - h)) / (2 * h)
            assert abs(float(K.grad) - dK) < 1e-7
            assert abs(float(a.grad) - dq1) < 1e-7
            assert abs(float(b.grad) - dq2) < 1e-7
            theta = math.acos(c)
            assert abs(float(K.grad) - (math.pi - theta) / (2 * math.pi)) < 1e-12
