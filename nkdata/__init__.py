"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module only draws inputs; it holds none of the kernel or solver
arithmetic.  The paper's datasets (CIFAR-10, CIFAR-5m, Tiny ImageNet) are not
available, so these generators stand in for them with the same shapes, class
counts and a short-range spatial correlation:

* images: i.i.d. N(0, 1) pixels, optionally blurred by a 3x3 box filter with
  zero padding (neighbouring pixels correlate as in natural images), then
  standardised per channel with the mean / std (ddof=0) of the TRAIN images,
  applied to train and test alike;
* FC inputs: N(0, 1) rows scaled to norm sqrt(d);
* labels: uniform random classes, one-hot minus 1/n_classes.

Generators are numpy PCG64 (``default_rng(seed)``); images are drawn in
float64 and cast once.  Seeds: 0 train, 1 test / target, 2 labels,
3 support initialisation, 4 Monte Carlo.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_TRAIN, SEED_TEST, SEED_LABELS, SEED_SUPPORT, SEED_MC = 0, 1, 2, 3, 4


def _box_blur(x: np.ndarray) -> np.ndarray:
    """3x3 mean with zero padding over (H, W) of x[N, H, W, C]."""
    n, h, w, c = x.shape
    p = np.zeros((n, h + 2, w + 2, c))
    p[:, 1:-1, 1:-1] = x
    out = np.zeros_like(x)
    for dy in range(3):
        for dx in range(3):
            out += p[:, dy:dy + h, dx:dx + w]
    return out / 9.0


def images(n: int, hw: int, c: int = 3, seed: int = SEED_TRAIN, blur: bool = True) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, hw, hw, c))
    if blur:
        x = _box_blur(x)
    return x


def standardise(train: np.ndarray, *others: np.ndarray):
    mu = train.mean(axis=(0, 1, 2), keepdims=True)
    sd = train.std(axis=(0, 1, 2), keepdims=True)
    outs = [(train - mu) / sd] + [(o - mu) / sd for o in others]
    return outs


def labels(n: int, n_classes: int, seed: int = SEED_LABELS) -> np.ndarray:
    rng = np.random.default_rng(seed)
    cls = rng.integers(0, n_classes, size=n)
    y = np.zeros((n, n_classes))
    y[np.arange(n), cls] = 1.0
    return y - 1.0 / n_classes


def fc_rows(n: int, d: int, seed: int = SEED_TRAIN) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    x *= np.sqrt(d) / np.linalg.norm(x, axis=1, keepdims=True)
    return x


def downsample2(x: np.ndarray) -> np.ndarray:
    """2x2 average of x[N, H, W, C] (the 32x32 companion of a 64x64 set)."""
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


@dataclass
class ImageProblem:
    x_train: np.ndarray
    x_test: np.ndarray
    y_train: np.ndarray
    y_test: np.ndarray


def image_problem(n_train: int, n_test: int, hw: int, n_classes: int = 10,
                  blur: bool = True, c: int = 3) -> ImageProblem:
    """Train/test images (seeds 0/1), standardised with train statistics, and
    labels (seed 2) for train followed by test."""
    tr = images(n_train, hw, c, SEED_TRAIN, blur)
    te = images(n_test, hw, c, SEED_TEST, blur)
    tr, te = standardise(tr, te)
    y = labels(n_train + n_test, n_classes, SEED_LABELS)
    return ImageProblem(tr, te, y[:n_train], y[n_train:])


# Workloads, named by network, image size and purpose (synthetic stand-ins
# with the shapes of the paper's experiments).
WORKLOADS = {
    "myrtle5_8x8_fp64": dict(hw=8, n_train=128, n_test=32, n_classes=10, blur=False, convs=(2, 1, 0),
                             sw2=2.0, sb2=0.0),
    "myrtle5_32x32": dict(hw=32, n_train=2048, n_test=512, n_classes=10, blur=True, convs=(2, 1, 0), sw2=2.0,
                          sb2=0.0),
    "myrtle10_32x32_grad": dict(hw=32, n_train=100, n_test=2048, n_classes=10, blur=True, convs=(3, 3, 3),
                                sw2=2.0, sb2=0.01),
    "fc3_3072": dict(d=3072, n_train=50000, n_test=10000, n_classes=10, sw2=2.0, sb2=0.01),
    "myrtle5_64x64_queue": dict(hw=64, n_train=512, n_test=128, n_classes=200, blur=True, convs=(2, 1, 0),
                                sw2=2.0, sb2=0.0),
}
