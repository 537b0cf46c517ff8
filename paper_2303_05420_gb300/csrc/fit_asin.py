"""Fit the arcsine polynomial used by the FP32 arc-cosine map in the kernels.

asin(m) = m + m^3 P(m^2) on m in [0, 1/sqrt(2)], P of degree ``DEG`` in
z = m^2.  The coefficients minimise the maximum relative error of asin(m)
(near-minimax: Lawson's iteratively re-weighted least squares on a dense
Chebyshev grid, float64).  Run ``python fit_asin.py`` to print the table that
``nk_map.cuh`` embeds, and the float64 error of the fit.
"""

import numpy as np

DEG = 6


def fit(deg=DEG, iters=400):
    zmax = 0.5
    t = np.cos(np.pi * (np.arange(4000) + 0.5) / 4000)
    z = (t + 1) * zmax / 2
    m = np.sqrt(z)
    f = np.arcsin(m)
    # relative error of asin: (m + m^3 P - f)/f -> weight m^3/f on residual of P
    target = (f - m) / (m ** 3)
    scale = m ** 3 / f
    V = np.vander(z, deg + 1, increasing=True)
    w = np.ones_like(z)
    for _ in range(iters):
        sw = np.sqrt(w) * scale
        c, *_ = np.linalg.lstsq(V * sw[:, None], target * sw, rcond=None)
        err = np.abs((V @ c - target) * scale)
        w = w * err
        w /= w.sum()
    return c


if __name__ == "__main__":
    c = fit()
    mm = np.linspace(1e-6, 2 ** -0.5, 200001)
    approx = mm + mm ** 3 * np.polyval(c[::-1], mm * mm)
    rel = np.abs(approx - np.arcsin(mm)) / np.arcsin(mm)
    print("max rel err (float64 eval): %.3e" % rel.max())
    for i, ci in enumerate(c):
        print("  %.9e,  // z^%d" % (ci, i))
