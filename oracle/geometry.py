"""Geometry-refinement losses of one view (Eq. 8-9) on a traced G-buffer, in
FP64 with PyTorch CPU autograd (TEST INFRASTRUCTURE ONLY, like the rest of
`oracle/`).

    L_D  = || C (D - D*) ||_1 / (|| C D* ||_1 + eps)                 (Eq. 8)
    L_N  = 1 - <N, N*>_F / (H W)                                      (Eq. 9)
    L_DN = 1 - <N^D, N*>_F / (H W)                                    (Eq. 9)

D is the rendered depth (ray distance of the composite), N the rendered,
renormalised normal, D* / C / N* the reference depth, its confidence and the
reference normals.  Readings of what the paper leaves open:
  - N^D, the depth-derived normal of pixel (x, y), is normalize(P_x x P_y)
    with P(q) = eye + D(q) d(q) the back-projected position along the pixel's
    ray d(q), P_x = P(x+1, y) - P(x-1, y) (image right) and
    P_y = P(x, y-1) - P(x, y+1) (image up), which faces the camera on a
    visible surface; it is 0 (no contribution) on the image border and where
    the pixel or one of its four neighbours has no composited hit;
  - both normal terms average over all H W pixels, as written.
Images are (H, W) row-major arrays (pixel p = y W + x); normals (H, W, 3).
"""
from __future__ import annotations

import numpy as np


def depth_normals(D, dirs, eye, valid):
    """N^D (H, W, 3) as torch FP64 tensors; D (H, W), dirs (H, W, 3), valid (H, W) bool."""
    import torch
    P = torch.as_tensor(eye, dtype=torch.float64).view(1, 1, 3) + D[..., None] * dirs
    H, W = D.shape
    N = torch.zeros((H, W, 3), dtype=torch.float64)
    px = P[1:-1, 2:] - P[1:-1, :-2]
    py = P[:-2, 1:-1] - P[2:, 1:-1]
    c = torch.cross(px, py, dim=-1)
    inner = c / torch.linalg.norm(c, dim=-1, keepdim=True).clamp_min(1e-300)
    ok = valid[1:-1, 1:-1] & valid[1:-1, 2:] & valid[1:-1, :-2] & valid[:-2, 1:-1] & valid[2:, 1:-1]
    N[1:-1, 1:-1] = torch.where(ok[..., None], inner, torch.zeros_like(inner))
    return N


def losses(depth, normal, dirs, hits, eye, depth_ref, conf, normal_ref, eps=1e-8, weights=(1.0, 1.0, 1.0)):
    """Returns (L_D, L_N, L_DN, dL/d depth (H, W), dL/d normal (H, W, 3)) for the
    weighted sum w_D L_D + w_N L_N + w_DN L_DN; inputs are numpy arrays."""
    import torch
    D = torch.tensor(np.asarray(depth, np.float64), requires_grad=True)
    N = torch.tensor(np.asarray(normal, np.float64), requires_grad=True)
    dirs_t = torch.tensor(np.asarray(dirs, np.float64))
    Ds = torch.tensor(np.asarray(depth_ref, np.float64))
    Cf = torch.tensor(np.asarray(conf, np.float64))
    Ns = torch.tensor(np.asarray(normal_ref, np.float64))
    valid = torch.as_tensor(np.asarray(hits) > 0)
    HW = D.numel()
    L_D = (Cf * (D - Ds)).abs().sum() / ((Cf * Ds).abs().sum() + eps)
    L_N = 1.0 - (N * Ns).sum() / HW
    ND = depth_normals(D, dirs_t, eye, valid)
    L_DN = 1.0 - (ND * Ns).sum() / HW
    total = weights[0] * L_D + weights[1] * L_N + weights[2] * L_DN
    total.backward()
    return (float(L_D.detach()), float(L_N.detach()), float(L_DN.detach()), D.grad.numpy().copy(),
            N.grad.numpy().copy())
