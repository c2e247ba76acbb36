"""Geometry-refinement losses (Eq. 8-9) on the GPU against the FP64 oracle:
the loss kernel on a seeded synthetic G-buffer (same inputs on both sides),
and the whole chain -- trace, loss, adjoint to the surfels -- on a room
scene, where each side renders its own G-buffer."""
import numpy as np
import pytest

import oracle
from oracle import geometry as OG
from synthetic import scenes as S
from tests._helpers import MG, flagged, gpu_tracer

pytestmark = pytest.mark.gpu


def _refs(rng, H, W, base=3.0):
    Ds = base + rng.normal(0, 0.2, (H, W))
    C = rng.uniform(0.0, 1.0, (H, W))
    Ns = np.concatenate([rng.normal(0, 0.3, (H, W, 2)), np.ones((H, W, 1))], -1)
    Ns /= np.linalg.norm(Ns, axis=-1, keepdims=True)
    return Ds.astype(np.float32), C.astype(np.float32), Ns.astype(np.float32)


def test_geometry_loss_kernel_matches_oracle_on_a_synthetic_gbuffer():
    import torch
    from paper_2608_29269_b300 import _native as N
    rng = np.random.default_rng(5)
    W, H = 67, 45
    cam = S.Camera((0.0, 0.2, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 55.0, W, H)
    dirs = oracle.camera_dirs(cam).reshape(H, W, 3).astype(np.float32)
    # a wavy surface in front of the camera: depth along each ray, with holes
    depth = (3.0 + 0.3 * np.sin(np.arange(W) / 7.0)[None, :] + 0.2 * np.cos(np.arange(H) / 5.0)[:, None]
             + rng.normal(0, 0.01, (H, W))).astype(np.float32)
    hits = (rng.uniform(size=(H, W)) > 0.03).astype(np.float32) * rng.integers(1, 9, (H, W))
    normal = rng.normal(0, 0.3, (H, W, 3)) + np.array([0.0, 0.0, 1.0])
    normal = (normal / np.linalg.norm(normal, axis=-1, keepdims=True)).astype(np.float32)
    Ds, C, Ns = _refs(rng, H, W)
    g = np.zeros((N.LF_GBUF_CHANNELS, H, W), np.float32)
    g[N.CH["depth"]] = depth
    g[N.CH["n"]:N.CH["n"] + 3] = normal.transpose(2, 0, 1)
    g[N.CH["hits"]] = hits
    g[N.CH["dir"]:N.CH["dir"] + 3] = dirs.transpose(2, 0, 1)
    tr, _ = gpu_tracer(S.scene_c1(0), [S.env_uniform(1.0, 8, 16)])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    dg = torch.zeros((N.LF_GBUF_CHANNELS, H, W), device="cuda")
    w = (0.7, 1.3, 0.9)
    L = tr.geometry_loss(cam, dev(g), dev(Ds), dev(C), dev(Ns.transpose(2, 0, 1)), 1e-8, w, dg)
    eye = np.array(cam.eye, np.float32).astype(np.float64)
    ref = OG.losses(depth, normal, dirs, hits, eye, Ds, C, Ns, 1e-8, w)
    print("losses gpu", L, "oracle", ref[:3])
    np.testing.assert_allclose(L, ref[:3], rtol=2e-6, atol=1e-7)
    dgh = dg.cpu().numpy()
    gD, gN = ref[3], ref[4]
    np.testing.assert_allclose(dgh[N.CH["depth"]], gD, rtol=1e-4, atol=2e-6 * np.abs(gD).max())
    np.testing.assert_allclose(dgh[N.CH["n"]:N.CH["n"] + 3].transpose(1, 2, 0), gN, rtol=1e-5, atol=1e-9)
    others = [c for c in range(N.LF_GBUF_CHANNELS) if c not in (N.CH["depth"], 6, 7, 8)]
    assert np.all(dgh[others] == 0)


def test_geometry_losses_through_the_tracer_and_adjoint():
    """Room scene: GPU G-buffer -> losses -> dL/dG -> adjoint to the surfels,
    against the oracle's G-buffer, its losses and its gradient.  Pixels whose
    3x3 neighbourhood holds a flagged primary decision get C = N* = 0 on both
    sides, so they and their stencils contribute nothing."""
    import torch
    from paper_2608_29269_b300 import _native as N
    sc = S.scene_c2(0, per_face=3000, per_object=8000)
    W = H = 48
    cam = S.camera_c2(W, H)
    env = S.env_uniform(1.0, 8, 16)
    tr, st = gpu_tracer(sc, [env])
    pix = np.arange(W * H, dtype=np.int32)
    o = oracle.render(sc, cam, env, pix, shade=False)
    flag = flagged(o["margins"]).reshape(H, W)
    pad = np.pad(flag, 1, constant_values=False)
    near = np.zeros_like(flag)
    for dy in (0, 1, 2):
        for dx in (0, 1, 2):
            near |= pad[dy:dy + H, dx:dx + W]
    rng = np.random.default_rng(7)
    Ds, C, Ns = _refs(rng, H, W, base=2.5)
    C[near] = 0.0
    Ns[near] = 0.0
    ch = o["ch"]
    OCH = {n: i for i, n in enumerate(oracle.CHANNELS)}
    depth = ch[:, OCH["depth"]].reshape(H, W)
    normal = ch[:, [OCH["n0"], OCH["n1"], OCH["n2"]]].reshape(H, W, 3)
    hits = ch[:, OCH["hits"]].reshape(H, W)
    dirs = oracle.camera_dirs(cam).reshape(H, W, 3)
    eye = np.array(cam.eye, np.float32).astype(np.float64)
    w = (1.0, 0.5, 2.0)
    ref = OG.losses(depth, normal, dirs, hits, eye, Ds, C, Ns, 1e-8, w)
    g_ch = np.zeros((W * H, oracle.NDIFF))
    g_ch[:, OCH["depth"]] = ref[3].reshape(-1)
    g_ch[:, [OCH["n0"], OCH["n1"], OCH["n2"]]] = ref[4].reshape(-1, 3)
    d_s, _ = oracle.grad(sc, cam, env, pix, 0, 0, None, g_ch, shade=False)
    g = tr.trace_primary(cam, 0)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    dg = torch.zeros((N.LF_GBUF_CHANNELS, H * W), device="cuda")
    L = tr.geometry_loss(cam, g, dev(Ds), dev(C), dev(Ns.transpose(2, 0, 1)), 1e-8, w, dg)
    print("losses gpu", L, "oracle", ref[:3], "near-flag pixels", int(near.sum()))
    np.testing.assert_allclose(L, ref[:3], rtol=1e-5, atol=1e-6)
    d_surf = torch.zeros((sc.n, 17), device="cuda")
    tr.backward(cam, g, 0, 1, 0, dL_dgbuf=dg, d_surfel=d_surf)
    tr.sync()
    gs = d_surf.cpu().numpy().astype(np.float64)
    for name, (a, b) in dict(mu=(0, 3), tu=(3, 6), tv=(6, 9), scale=(9, 11), opacity=(11, 12)).items():
        r_, g_ = d_s[:, a:b], gs[:, a:b]
        rel = np.linalg.norm(g_ - r_) / np.linalg.norm(r_)
        print("geometry adjoint", name, "L2-relative", rel)
        assert rel <= 1e-3, name
    assert np.abs(gs[:, 12:]).max() == 0.0  # materials take no geometry gradient
