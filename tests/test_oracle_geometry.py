"""Pins of the oracle's geometry-refinement losses (Eq. 8-9) to closed forms:
identical maps give zero loss, a uniform depth offset and a uniform normal
rotation give known values, a plane seen by a pinhole camera has the plane's
normal as its depth-derived normal, and the autograd gradients match central
finite differences of the loss."""
import numpy as np
import pytest

import oracle
from oracle import geometry as G
from synthetic.scenes import Camera

pytest.importorskip("torch")


def _plane_view(normal, point, W=24, H=20):
    cam = Camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 50.0, W, H)
    d = oracle.camera_dirs(cam).reshape(H, W, 3)
    eye = np.array(cam.eye, np.float64)
    n = np.asarray(normal, np.float64) / np.linalg.norm(normal)
    t = ((np.asarray(point, np.float64) - eye) @ n) / (d @ n)  # ray distance to the plane
    return cam, eye, d, t, n


def test_identical_maps_give_zero_depth_and_normal_loss():
    rng = np.random.default_rng(0)
    H, W = 8, 9
    D = rng.uniform(1, 3, (H, W))
    N = rng.normal(size=(H, W, 3))
    N /= np.linalg.norm(N, axis=-1, keepdims=True)
    dirs = np.tile([0.0, 0.0, -1.0], (H, W, 1))
    L_D, L_N, _, _, _ = G.losses(D, N, dirs, np.ones((H, W)), np.zeros(3), D, np.ones((H, W)), N)
    assert L_D == 0.0 and abs(L_N) < 1e-15


def test_uniform_depth_offset_and_normal_rotation_closed_forms():
    H, W = 6, 7
    rng = np.random.default_rng(1)
    Ds = rng.uniform(1, 2, (H, W))
    C = rng.uniform(0, 1, (H, W))
    dirs = np.tile([0.0, 0.0, -1.0], (H, W, 1))
    Ns = np.tile([0.0, 0.0, 1.0], (H, W, 1))
    th = 0.3
    N = np.tile([np.sin(th), 0.0, np.cos(th)], (H, W, 1))
    L_D, L_N, _, _, _ = G.losses(Ds + 0.25, N, dirs, np.ones((H, W)), np.zeros(3), Ds, C, Ns, eps=0.0)
    assert abs(L_D - 0.25 * C.sum() / (C * Ds).sum()) < 1e-14
    assert abs(L_N - (1.0 - np.cos(th))) < 1e-14


@pytest.mark.parametrize("normal", [(0.0, 0.0, 1.0), (0.3, -0.2, 1.0), (-0.5, 0.4, 0.8)])
def test_depth_derived_normal_of_a_plane_is_the_plane_normal(normal):
    cam, eye, d, t, n = _plane_view(normal, (0.1, -0.05, 0.2))
    H, W = t.shape
    ND = G.depth_normals(__import__("torch").as_tensor(t), __import__("torch").as_tensor(d), eye,
                         __import__("torch").ones((H, W), dtype=bool)).numpy()
    inner = ND[1:-1, 1:-1]
    np.testing.assert_allclose(inner, np.broadcast_to(n, inner.shape), atol=1e-7)  # FP32-rounded rays
    assert np.all(ND[0] == 0) and np.all(ND[:, -1] == 0)
    # with N* = the plane normal, L_DN = 1 - (interior pixels) / (H W)
    _, _, L_DN, _, _ = G.losses(t, np.broadcast_to(n, (H, W, 3)), d, np.ones((H, W)), eye, t, np.ones((H, W)),
                                np.broadcast_to(n, (H, W, 3)))
    assert abs(L_DN - (1.0 - (H - 2) * (W - 2) / (H * W))) < 1e-7


def test_missing_hits_drop_their_neighbourhood_from_the_depth_normals():
    cam, eye, d, t, n = _plane_view((0.0, 0.0, 1.0), (0.0, 0.0, 0.0), W=10, H=9)
    hits = np.ones(t.shape)
    hits[4, 5] = 0
    import torch
    ND = G.depth_normals(torch.as_tensor(t), torch.as_tensor(d), eye, torch.as_tensor(hits > 0)).numpy()
    for (y, x) in [(4, 5), (3, 5), (5, 5), (4, 4), (4, 6)]:
        assert np.all(ND[y, x] == 0)
    assert np.linalg.norm(ND[2, 2]) > 0.99


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    cam, eye, d, t, n = _plane_view((0.2, 0.1, 1.0), (0.0, 0.0, 0.0), W=7, H=6)
    H, W = t.shape
    D = t + rng.normal(0, 0.02, t.shape)
    N = np.broadcast_to(n, (H, W, 3)) + rng.normal(0, 0.1, (H, W, 3))
    N /= np.linalg.norm(N, axis=-1, keepdims=True)
    Ds, C = t + rng.normal(0, 0.05, t.shape), rng.uniform(0.2, 1, t.shape)
    Ns = np.broadcast_to(n, (H, W, 3)) + rng.normal(0, 0.2, (H, W, 3))
    Ns /= np.linalg.norm(Ns, axis=-1, keepdims=True)
    hits = np.ones((H, W))
    w = (0.7, 1.3, 0.9)
    f = lambda D_, N_: sum(wi * li for wi, li in zip(w, G.losses(D_, N_, d, hits, eye, Ds, C, Ns, 1e-8, w)[:3]))
    _, _, _, gD, gN = G.losses(D, N, d, hits, eye, Ds, C, Ns, 1e-8, w)
    h = 1e-6
    for (y, x) in [(2, 3), (1, 1), (4, 5), (0, 0)]:
        Dp, Dm = D.copy(), D.copy()
        Dp[y, x] += h
        Dm[y, x] -= h
        assert abs((f(Dp, N) - f(Dm, N)) / (2 * h) - gD[y, x]) < 1e-6
        for k in range(3):
            Np, Nm = N.copy(), N.copy()
            Np[y, x, k] += h
            Nm[y, x, k] -= h
            assert abs((f(D, Np) - f(D, Nm)) / (2 * h) - gN[y, x, k]) < 1e-6
