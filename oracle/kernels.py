"""Oracle kernels: ReLU arc-cosine map, Myrtle CNN NNGP recursion, FC3 NNGP.

Test infrastructure only (see the package docstring).  Everything is float64
torch on the CPU, written as the plain definition with no blocking or fusion.

Notation: an image is x[H, W, C]; a pixel p = (i, j); K_l(p, p') is a
pre-activation covariance and Kt_l(p, p') a post-activation covariance; the
pixel-pair tensor of a pair (x, x') is stored as K[i, j, i', j'].
"""

from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import torch

F64 = torch.float64


@dataclass(frozen=True)
class Arch:
    """Myrtle-family architecture (Appendix A, Myrtle listing).

    ``convs[s]`` conv(3x3, SAME)+activation layers in stage s; a 2x2 stride-2
    average pool sits between consecutive stages; the last stage ends in a
    global average pool and a Dense readout.  Myrtle-10 is (3, 3, 3) (the
    listing: one conv, two more, pool, three, pool, three, GAP, Dense; the
    first stage therefore holds three convs).  ``filt`` is the square filter
    size (3 in the paper; 1 is used by a test reduction).  ``act`` is "relu"
    (the paper's Myrtle listings), "erf" (one of the activations of the
    paper's architecture search, Appendix on tuning the Myrtle architecture)
    or "identity" (a test-only linear network).  ``norm`` is "none" (the
    Myrtle listings) or "layer": a LayerNorm over every axis of each image's
    hidden representation (pixels and channels, as in the tuned Myrtle
    listing) between each conv and its activation.  At infinite width the
    channel mean of a centred pre-activation vanishes and its mean square over
    pixels and channels tends to m = mean_p q(p), so the normalised covariance
    is K(p, p') / sqrt(m m') and the normalised self-variances q / m.
    """

    convs: Tuple[int, ...] = (2, 1, 0)
    filt: int = 3
    act: str = "relu"
    norm: str = "none"

    @property
    def n_weight_layers(self) -> int:
        return sum(self.convs) + 1


# --------------------------------------------------------------------------
# ReLU arc-cosine map (stax.Relu in the Appendix A listings)
# --------------------------------------------------------------------------


class _ArccosJ(torch.autograd.Function):
    """J(c) = sin(theta) + (pi - theta) cos(theta), theta = arccos(c).

    The degree-1 arc-cosine kernel: E[relu(u) relu(v)] = sqrt(q q')/(2 pi) J(c)
    for (u, v) centred Gaussian with variances q, q' and correlation c.  Its
    derivative is J'(c) = pi - arccos(c), finite on [-1, 1]; autograd through
    arccos and sqrt would give inf * 0 at c = +-1, so the derivative is stated
    here in closed form.
    """

    @staticmethod
    def forward(ctx, c):
        ctx.save_for_backward(c)
        theta = torch.arccos(c)
        return torch.sqrt(torch.clamp(1.0 - c * c, min=0.0)) + (math.pi - theta) * c

    @staticmethod
    def backward(ctx, g):
        (c,) = ctx.saved_tensors
        return g * (math.pi - torch.arccos(c))


def arccos_J(c: torch.Tensor) -> torch.Tensor:
    return _ArccosJ.apply(c)


def relu_map(K: torch.Tensor, q1: torch.Tensor, q2: torch.Tensor) -> torch.Tensor:
    """Post-ReLU covariance from pre-activation covariance K and variances q1, q2.

    Kt = sqrt(q1 q2) / (2 pi) * J(c), c = clamp(K / sqrt(q1 q2), -1, 1);
    Kt = 0 where q1 q2 = 0 (a zero-variance input gives a zero output).
    """
    s = torch.sqrt(q1 * q2)
    pos = s > 0
    s_safe = torch.where(pos, s, torch.ones_like(s))
    c = torch.clamp(K / s_safe, -1.0, 1.0)
    out = s_safe / (2.0 * math.pi) * arccos_J(c)
    return torch.where(pos, out, torch.zeros_like(out))


# --------------------------------------------------------------------------
# Erf map (stax.Erf: the activation erf(x))
# --------------------------------------------------------------------------


def erf_map(K: torch.Tensor, q1: torch.Tensor, q2: torch.Tensor) -> torch.Tensor:
    """E[erf(u) erf(v)] for centred Gaussians (u, v) with variances q1, q2 and
    covariance K: (2 / pi) arcsin(2 K / sqrt((1 + 2 q1)(1 + 2 q2))), the
    closed form of the Gaussian integral of the error function (Williams,
    1997).  Zero at K = 0; the argument stays inside [-1, 1] because
    |K| <= sqrt(q1 q2)."""
    return (2.0 / math.pi) * torch.arcsin(2.0 * K / torch.sqrt((1.0 + 2.0 * q1) * (1.0 + 2.0 * q2)))


def erf_derivative_map(K: torch.Tensor, q1: torch.Tensor, q2: torch.Tensor) -> torch.Tensor:
    """E[erf'(u) erf'(v)], erf'(x) = (2 / sqrt(pi)) exp(-x^2), for centred
    Gaussians with variances q1, q2 and covariance K:
    (4 / pi) / sqrt((1 + 2 q1)(1 + 2 q2) - 4 K^2)."""
    return (4.0 / math.pi) / torch.sqrt((1.0 + 2.0 * q1) * (1.0 + 2.0 * q2) - 4.0 * K * K)


def _activate(arch: Arch, K, q1, q2):
    if arch.act == "relu":
        return relu_map(K, q1, q2)
    if arch.act == "erf":
        return erf_map(K, q1, q2)
    if arch.act == "identity":
        return K
    raise ValueError(arch.act)


# --------------------------------------------------------------------------
# Pixel-pair tensor operations
# --------------------------------------------------------------------------


def input_cov(x: torch.Tensor, xp: torch.Tensor) -> torch.Tensor:
    """K_0(p, p') = (1/C) sum_c x[p, c] x'[p', c]  (first conv has fan_in C k^2)."""
    C = x.shape[-1]
    return torch.einsum("ijc,klc->ijkl", x, xp) / C


def conv_pp(Kt: torch.Tensor, sw2, sb2, filt: int) -> torch.Tensor:
    """SAME conv on both pixel indices (stax.Conv, padding='SAME').

    K_next(p, p') = sw2 / filt^2 * sum_delta Kt(p + delta, p' + delta) + sb2,
    a term being zero when p + delta or p' + delta leaves its image.  The
    divisor stays filt^2 at the borders because fan_in = C * filt^2 for every
    output position.
    """
    r = filt // 2
    H, W, H2, W2 = Kt.shape[-4:]
    pad = torch.nn.functional.pad(Kt, (r, r, r, r, r, r, r, r))
    acc = torch.zeros_like(Kt)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            acc = acc + pad[..., r + dy:r + dy + H, r + dx:r + dx + W,
                            r + dy:r + dy + H2, r + dx:r + dx + W2]
    return sw2 / (filt * filt) * acc + sb2


def avgpool_pp(Kt: torch.Tensor) -> torch.Tensor:
    """stax.AvgPool((2, 2), strides=(2, 2)) on both images:
    K(P, P') = 1/16 sum_{a, b in {0,1}^2} Kt(2P + a, 2P' + b)."""
    H, W, H2, W2 = Kt.shape[-4:]
    if H % 2 or W % 2 or H2 % 2 or W2 % 2:
        raise ValueError("2x2 VALID pooling of an odd-sized image")
    lead = Kt.shape[:-4]
    v = Kt.reshape(*lead, H // 2, 2, W // 2, 2, H2 // 2, 2, W2 // 2, 2)
    n = len(lead)
    return v.mean(dim=(n + 1, n + 3, n + 5, n + 7))


def _diag(K: torch.Tensor) -> torch.Tensor:
    H, W = K.shape[-4], K.shape[-3]
    return torch.diagonal(K.reshape(*K.shape[:-4], H * W, H * W), dim1=-2, dim2=-1).reshape(
        *K.shape[:-4], H, W)


# --------------------------------------------------------------------------
# Myrtle recursion
# --------------------------------------------------------------------------


def myrtle_layers_pair(arch: Arch, sw2, sb2, x, xp,
                       q_x: Optional[List[torch.Tensor]] = None,
                       q_xp: Optional[List[torch.Tensor]] = None):
    """Run the Myrtle NNGP recursion on the pair (x, x').

    ``q_x`` / ``q_xp``: per-activation-layer self-variances q_l(p) of x and x'
    (lists of [H_l, W_l] tensors, as returned by :func:`myrtle_self_q`).  When
    both are None the pair must be a self pair (x is x') and q is read off the
    diagonal of the running tensor.

    Returns (K, qs, pre) with K the kernel value (Appendix A readout:
    Dense(W_std, b_std) after GlobalAvgPool: K = sw2 * mean Kt + sb2), qs the
    list of self-variances of each conv's output (before a LayerNorm) and pre
    the list of the activations' input tensors.
    """
    self_pair = q_x is None
    qs: List[torch.Tensor] = []
    pre: List[torch.Tensor] = []
    Kt = input_cov(x, xp)
    li = 0
    for s, n in enumerate(arch.convs):
        if s > 0:
            Kt = avgpool_pp(Kt)
        for _ in range(n):
            K = conv_pp(Kt, sw2, sb2, arch.filt)
            if self_pair:
                q = _diag(K)
                q1, q2 = q, q
            else:
                q1, q2 = q_x[li], q_xp[li]
            qs.append(q1)
            if arch.norm == "layer":
                m1, m2 = q1.mean(), q2.mean()
                K = K / torch.sqrt(m1 * m2)
                q1, q2 = q1 / m1, q2 / m2
            elif arch.norm != "none":
                raise ValueError(arch.norm)
            pre.append(K)
            Kt = _activate(arch, K, q1[:, :, None, None], q2[None, None, :, :])
            li += 1
    K = sw2 * Kt.mean(dim=(-4, -3, -2, -1)) + sb2
    return K, qs, pre


def relu_derivative_map(K: torch.Tensor, q1: torch.Tensor, q2: torch.Tensor) -> torch.Tensor:
    """E[relu'(u) relu'(v)] for centred Gaussians with variances q1, q2 and
    covariance K: (pi - arccos c) / (2 pi), c = clamp(K / sqrt(q1 q2), -1, 1);
    zero where q1 q2 = 0."""
    s = torch.sqrt(q1 * q2)
    pos = s > 0
    s_safe = torch.where(pos, s, torch.ones_like(s))
    c = torch.clamp(K / s_safe, -1.0, 1.0)
    out = (math.pi - torch.arccos(c)) / (2.0 * math.pi)
    return torch.where(pos, out, torch.zeros_like(out))


def myrtle_ntk_pair(arch: Arch, sw2, sb2, x, xp, q_x: List[torch.Tensor], q_xp: List[torch.Tensor]):
    """NNGP K and neural tangent kernel Theta of the Myrtle network on the
    pair (x, x'), in the NTK parameterisation of the Appendix A listings
    (stax's default: every weight and bias is a standard normal scaled in the
    forward pass).  Differentiating the output with respect to the parameters
    of a layer gives that layer's NNGP term, and the chain rule through a
    ReLU multiplies by the derivative kernel, so:
      input      Theta_0 = 0
      conv       K' = sw2 A(Kt) + sb2,  Theta' = K' + sw2 A(Theta_t)
                 (A the 3x3 SAME average on both pixels, divisor 9)
      ReLU       Kt = relu_map(K),  Theta_t = Theta * E[relu' relu']
      Erf        Kt = erf_map(K),   Theta_t = Theta * E[erf' erf']
      identity   Kt = K,  Theta_t = Theta
      avg pool   the same linear pool on both
      readout    K = sw2 mean Kt + sb2,  Theta = K + sw2 mean Theta_t.
    Returns (K, Theta)."""
    Kt = input_cov(x, xp)
    Tt = torch.zeros_like(Kt)
    li = 0
    for s, n in enumerate(arch.convs):
        if s > 0:
            Kt = avgpool_pp(Kt)
            Tt = avgpool_pp(Tt)
        for _ in range(n):
            K = conv_pp(Kt, sw2, sb2, arch.filt)
            T = K + conv_pp(Tt, sw2, 0.0, arch.filt)
            q1, q2 = q_x[li][:, :, None, None], q_xp[li][None, None, :, :]
            if arch.norm == "layer":
                # a deterministic per-image scale in the limit: K and Theta alike
                m1, m2 = q_x[li].mean(), q_xp[li].mean()
                K, T = K / torch.sqrt(m1 * m2), T / torch.sqrt(m1 * m2)
                q1, q2 = q1 / m1, q2 / m2
            if arch.act == "relu":
                Kt = relu_map(K, q1, q2)
                Tt = T * relu_derivative_map(K, q1, q2)
            elif arch.act == "erf":
                Kt = erf_map(K, q1, q2)
                Tt = T * erf_derivative_map(K, q1, q2)
            elif arch.act == "identity":
                Kt, Tt = K, T
            else:
                raise ValueError(arch.act)
            li += 1
    Kout = sw2 * Kt.mean(dim=(-4, -3, -2, -1)) + sb2
    Tout = Kout + sw2 * Tt.mean(dim=(-4, -3, -2, -1))
    return Kout, Tout


def myrtle_ntk_block(arch: Arch, sw2, sb2, Xa, Xb) -> Tuple[torch.Tensor, torch.Tensor]:
    """(K, Theta) blocks for all pairs of Xa x Xb."""
    Xa = torch.as_tensor(Xa, dtype=F64)
    Xb = torch.as_tensor(Xb, dtype=F64)
    qa = [myrtle_self_q(arch, sw2, sb2, x) for x in Xa]
    qb = [myrtle_self_q(arch, sw2, sb2, x) for x in Xb]
    K = torch.zeros((Xa.shape[0], Xb.shape[0]), dtype=F64)
    T = torch.zeros_like(K)
    for i in range(Xa.shape[0]):
        for j in range(Xb.shape[0]):
            K[i, j], T[i, j] = myrtle_ntk_pair(arch, sw2, sb2, Xa[i], Xb[j], qa[i], qb[j])
    return K, T


def myrtle_self_q(arch: Arch, sw2, sb2, x) -> List[torch.Tensor]:
    """Self-variances q_l(p) = K_l(p, p; x, x) at every activation layer,
    read off the diagonal of the FULL self tensor (no band)."""
    _, qs, _ = myrtle_layers_pair(arch, sw2, sb2, x, x)
    return qs


def myrtle_pair(arch: Arch, sw2, sb2, x, xp) -> torch.Tensor:
    qx = myrtle_self_q(arch, sw2, sb2, x)
    qxp = myrtle_self_q(arch, sw2, sb2, xp)
    K, _, _ = myrtle_layers_pair(arch, sw2, sb2, x, xp, qx, qxp)
    return K


def myrtle_block(arch: Arch, sw2, sb2, Xa, Xb, symmetric: bool = False,
                 pairs: Optional[Sequence[Tuple[int, int]]] = None) -> torch.Tensor:
    """Kernel block K[i, j] = NNGP(Xa[i], Xb[j]) (Figure 1 top: blocks of the
    kernel matrix are independent).  ``pairs`` restricts the evaluation to the
    listed (i, j); other entries are NaN.  ``symmetric`` evaluates i <= j and
    mirrors (Xa and Xb must then be the same set)."""
    Xa = torch.as_tensor(Xa, dtype=F64)
    Xb = torch.as_tensor(Xb, dtype=F64)
    qa = [myrtle_self_q(arch, sw2, sb2, x) for x in Xa]
    qb = qa if symmetric else [myrtle_self_q(arch, sw2, sb2, x) for x in Xb]
    out = torch.full((Xa.shape[0], Xb.shape[0]), float("nan"), dtype=F64)
    if pairs is None:
        pairs = [(i, j) for i in range(Xa.shape[0]) for j in range(Xb.shape[0])
                 if (not symmetric or i <= j)]
    for i, j in pairs:
        K, _, _ = myrtle_layers_pair(arch, sw2, sb2, Xa[i], Xb[j], qa[i], qb[j])
        out[i, j] = K
        if symmetric:
            out[j, i] = K
    return out


# --------------------------------------------------------------------------
# FC3 (Appendix A, FC listing)
# --------------------------------------------------------------------------


def cv_pair(sw2, sb2, x, xp, depth: int = 8, filt: int = 3, act: str = "relu") -> torch.Tensor:
    """NNGP of the CV8 listing (Appendix A): ``depth`` conv(filt x filt, SAME)
    + activation layers, then Flatten and a Dense readout.  The readout's
    weights are independent per position, so only the diagonal of the last
    post-activation tensor enters: K = sw2 mean_p Kt_L(p, p) + sb2.  The
    whole pixel-pair tensor is carried through every layer (the plain
    definition); self-variances from the full self tensors."""
    arch = Arch((depth,), filt, act)
    x = torch.as_tensor(x, dtype=F64)
    xp = torch.as_tensor(xp, dtype=F64)
    qx = myrtle_self_q(arch, sw2, sb2, x)
    qxp = myrtle_self_q(arch, sw2, sb2, xp)
    Kt = input_cov(x, xp)
    for layer in range(depth):
        K = conv_pp(Kt, sw2, sb2, filt)
        Kt = _activate(arch, K, qx[layer][:, :, None, None], qxp[layer][None, None, :, :])
    H, W = Kt.shape[0], Kt.shape[1]
    i = torch.arange(H)[:, None]
    j = torch.arange(W)[None, :]
    return sw2 * Kt[i, j, i, j].mean() + sb2


def cv_block(Xa, Xb, sw2, sb2, depth: int = 8, filt: int = 3, act: str = "relu") -> torch.Tensor:
    """CV8-style NNGP for all pairs of Xa x Xb."""
    Xa = torch.as_tensor(Xa, dtype=F64)
    Xb = torch.as_tensor(Xb, dtype=F64)
    K = torch.zeros((Xa.shape[0], Xb.shape[0]), dtype=F64)
    for a in range(Xa.shape[0]):
        for b in range(Xb.shape[0]):
            K[a, b] = cv_pair(sw2, sb2, Xa[a], Xb[b], depth, filt, act)
    return K


def fc_nngp(X1, X2, sw2, sb2, depth: int = 3, act: str = "relu") -> torch.Tensor:
    """FC NNGP: K_0 = x.x'/d; K = sw2 K_0 + sb2; then ``depth`` times
    K <- sw2 * relu_map(K) + sb2 (Dense(512)+Relu x depth, Dense readout)."""
    X1 = torch.as_tensor(X1, dtype=F64)
    X2 = torch.as_tensor(X2, dtype=F64)
    d = X1.shape[1]
    K = X1 @ X2.T / d
    q1 = (X1 * X1).sum(1) / d
    q2 = (X2 * X2).sum(1) / d
    K = sw2 * K + sb2
    q1 = sw2 * q1 + sb2
    q2 = sw2 * q2 + sb2
    for _ in range(depth):
        if act == "relu":
            K = sw2 * relu_map(K, q1[:, None], q2[None, :]) + sb2
            q1 = sw2 * relu_map(q1, q1, q1) + sb2
            q2 = sw2 * relu_map(q2, q2, q2) + sb2
        else:
            K = sw2 * K + sb2
            q1 = sw2 * q1 + sb2
            q2 = sw2 * q2 + sb2
    return K
