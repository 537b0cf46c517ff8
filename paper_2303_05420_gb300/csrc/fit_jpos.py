"""Fit the polynomial of the FP32 arc-cosine map on c in [0, 1].

J(c) = sqrt(1 - c^2) + c (pi - arccos c) = pi c + (1 - c)^{3/2} B(c), with B
analytic on [0, 1] (its nearest singularity is at c = -1; B(1) = 2 sqrt(2)/3).
B is approximated by a polynomial of degree ``DEG`` minimising the maximum
ABSOLUTE error of J (Lawson's iteratively re-weighted least squares on a dense
Chebyshev grid); targets are computed with 40-digit mpmath through
theta = arccos c, J - pi c = sin(theta) - theta cos(theta), to avoid the
cancellation near c = 1.  For c in [-1, 0) the map uses
J(c) = J(|c|) + pi min(c, 0).  Run ``python fit_jpos.py`` to print the table
that nk_map.cuh embeds.
"""

import mpmath as mp
import numpy as np

DEG = 5
mp.mp.dps = 40


def target(c):
    c = mp.mpf(c)
    if c == 1:
        return 2 * mp.sqrt(2) / 3
    t = mp.acos(c)
    return (mp.sin(t) - t * mp.cos(t)) / (1 - c) ** mp.mpf(1.5)


def fit(deg=DEG, n=3000, iters=300):
    x = (np.cos(np.pi * (np.arange(n) + 0.5) / n) + 1) / 2
    B = np.array([float(target(v)) for v in x])
    wgt = (1 - x) ** 1.5
    V = np.vander(x, deg + 1, increasing=True)
    w = np.ones(n)
    for _ in range(iters):
        sw = np.sqrt(w) * wgt
        c, *_ = np.linalg.lstsq(V * sw[:, None], B * sw, rcond=None)
        err = np.abs((V @ c - B) * wgt)
        w = w * (err + 1e-30)
        w /= w.sum()
    return c


if __name__ == "__main__":
    c = fit()
    xs = np.linspace(0, 1, 20001)
    Jt = np.array([float(mp.pi * v + (1 - mp.mpf(v)) ** mp.mpf(1.5) * target(v)) for v in xs[::20]])
    Ja = np.pi * xs[::20] + (1 - xs[::20]) ** 1.5 * np.polyval(c[::-1], xs[::20])
    print("max abs err of J (float64 eval): %.3e" % np.abs(Ja - Jt).max())
    for i, ci in enumerate(c):
        print("  %.9e,  // c^%d" % (ci, i))
