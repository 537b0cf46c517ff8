"""Oracle kernel-ridge support-set loss and its gradients.

Test infrastructure only.  With support images X_s (labels Y_s) and target
images X_t (labels Y_t):

    A = (K_ss + lam I)^{-1} Y_s,  Yhat = K_ts A,  L = 1/2 mean((Yhat - Y_t)^2)

(kernel-ridge prediction as in Section 2; the loss is the benchmark's choice).
lam is held fixed under differentiation.  Gradients w.r.t. sigma_w^2,
sigma_b^2 and X_s come from torch autograd through the float64 definition in
``kernels.py``; they are checked in tests against central differences.
"""

from __future__ import annotations

import torch

from .kernels import Arch, myrtle_layers_pair, myrtle_self_q

F64 = torch.float64


def _kernel_blocks(arch: Arch, sw2, sb2, Xs, Xt):
    qs = [myrtle_self_q(arch, sw2, sb2, x) for x in Xs]
    qt = [myrtle_self_q(arch, sw2, sb2, x) for x in Xt]
    ns, nt = Xs.shape[0], Xt.shape[0]
    Kss = [[None] * ns for _ in range(ns)]
    for i in range(ns):
        for j in range(i, ns):
            k, _, _ = myrtle_layers_pair(arch, sw2, sb2, Xs[i], Xs[j], qs[i], qs[j])
            Kss[i][j] = k
            Kss[j][i] = k
    Kts = [[myrtle_layers_pair(arch, sw2, sb2, Xt[a], Xs[j], qt[a], qs[j])[0]
            for j in range(ns)] for a in range(nt)]
    Kss = torch.stack([torch.stack(r) for r in Kss])
    Kts = torch.stack([torch.stack(r) for r in Kts])
    return Kss, Kts


def krr_loss(arch: Arch, sw2, sb2, Xs, Ys, Xt, Yt, lam: float):
    Xs = torch.as_tensor(Xs, dtype=F64)
    Xt = torch.as_tensor(Xt, dtype=F64)
    Ys = torch.as_tensor(Ys, dtype=F64)
    Yt = torch.as_tensor(Yt, dtype=F64)
    Kss, Kts = _kernel_blocks(arch, sw2, sb2, Xs, Xt)
    n = Kss.shape[0]
    A = torch.linalg.solve(Kss + lam * torch.eye(n, dtype=F64), Ys)
    Yhat = Kts @ A
    return 0.5 * ((Yhat - Yt) ** 2).mean()


def krr_loss_and_grads(arch: Arch, sw2: float, sb2: float, Xs, Ys, Xt, Yt, lam: float):
    """Returns (L, dL/dsw2, dL/dsb2, dL/dXs) in float64."""
    sw2_t = torch.tensor(float(sw2), dtype=F64, requires_grad=True)
    sb2_t = torch.tensor(float(sb2), dtype=F64, requires_grad=True)
    Xs_t = torch.as_tensor(Xs, dtype=F64).clone().requires_grad_(True)
    L = krr_loss(arch, sw2_t, sb2_t, Xs_t, Ys, Xt, Yt, lam)
    L.backward()
    return float(L.detach()), float(sw2_t.grad), float(sb2_t.grad), Xs_t.grad.detach().clone()
