"""Regularisers of the training objectives, in FP64 with PyTorch CPU autograd
(TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`).

    L_alpha = || A - 1 ||_1 / (H W)                                   (Eq. 4)
    L_s     = (1/N) sum_i max(0, ||s_i||_inf / s_max - 1)^2            (Eq. 5)
    L_TV(E) = total variation of an environment map                   (Eq. 14)

Readings of what the paper leaves open:
  - in the ray-traced objectives A is the traced accumulated opacity, the
    composite's weight sum W = sum_j w_j (= 1 - T) of each pixel;
  - at a tie of the two scales, ||s||_inf passes its gradient to both halves
    equally;
  - L_TV is the anisotropic L1 total variation averaged over the texels and
    colour channels, (1 / (3 H W)) sum |E(r, c+1) - E(r, c)| + |E(r+1, c) - E(r, c)|,
    wrapping in the azimuthal (column) direction and not across the poles
    (rows).
"""
from __future__ import annotations

import numpy as np


def opacity_loss(W):
    """(L_alpha, dL/dW) for the (H, W) weight-sum map."""
    import torch
    Wt = torch.tensor(np.asarray(W, np.float64), requires_grad=True)
    L = (Wt - 1.0).abs().sum() / Wt.numel()
    L.backward()
    return float(L.detach()), Wt.grad.numpy().copy()


def scale_loss(scale, s_max):
    """(L_s, dL/d scale) for the (N, 2) in-plane scales."""
    import torch
    s = torch.tensor(np.asarray(scale, np.float64), requires_grad=True)
    L = (torch.clamp(s.amax(dim=1) / s_max - 1.0, min=0.0) ** 2).mean()
    L.backward()
    return float(L.detach()), s.grad.numpy().copy()


def env_tv(E):
    """(L_TV, dL/dE) for an (H, W, 3) environment map."""
    import torch
    Et = torch.tensor(np.asarray(E, np.float64), requires_grad=True)
    du = (torch.roll(Et, -1, dims=1) - Et).abs().sum()
    dv = (Et[1:] - Et[:-1]).abs().sum()
    L = (du + dv) / Et.numel()
    L.backward()
    return float(L.detach()), Et.grad.numpy().copy()
