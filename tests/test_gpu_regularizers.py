"""Regularisers (Eq. 4, 5, 14) on the GPU against the FP64 oracle: the same
seeded inputs on both sides, and the opacity term through the adjoint."""
import numpy as np
import pytest

import oracle
from oracle import regularizers as OR
from synthetic import scenes as S
from tests._helpers import gpu_tracer

pytestmark = pytest.mark.gpu


def test_scale_and_env_tv_match_oracle():
    import torch
    sc = S.scene_c1(0)
    rng = np.random.default_rng(2)
    smax = 0.06
    sc.scale[:] = rng.uniform(0.01, 0.1, sc.scale.shape).astype(np.float32)
    sc.scale[7] = [0.08, 0.08]  # a tie above s_max
    tr, st = gpu_tracer(sc, [S.env_uniform(1.0, 8, 16)])
    d_surf = torch.zeros((sc.n, 17), device="cuda")
    L = tr.scale_loss(smax, 0.5, d_surf)
    Lr, g = OR.scale_loss(sc.scale, smax)
    assert abs(L - Lr) <= 1e-6 * Lr
    got = d_surf.cpu().numpy()
    np.testing.assert_allclose(got[:, 9:11], 0.5 * g, rtol=1e-5, atol=1e-9)
    assert np.all(got[:, :9] == 0) and np.all(got[:, 11:] == 0)
    env = S.env_sky_sun(3, 32, 64)
    E = torch.as_tensor(env.rgb, device="cuda").contiguous()
    d_env = torch.zeros_like(E)
    L = tr.env_tv_loss(E, 2.0, d_env)
    Lr, g = OR.env_tv(env.rgb)
    assert abs(L - Lr) <= 1e-6 * Lr
    np.testing.assert_allclose(d_env.cpu().numpy(), 2.0 * g, rtol=1e-6, atol=1e-12)


def test_opacity_loss_matches_oracle_and_flows_through_the_adjoint():
    import torch
    from paper_2608_29269_b300 import _native as N
    sc = S.scene_c2(0, per_face=3000, per_object=8000)
    W = H = 48
    cam = S.camera_c2(W, H)
    env = S.env_uniform(1.0, 8, 16)
    tr, _ = gpu_tracer(sc, [env])
    g = tr.trace_primary(cam, 0)
    dg = torch.zeros((N.LF_GBUF_CHANNELS, H * W), device="cuda")
    L = tr.opacity_loss(cam, g, 1.5, dg)
    pix = np.arange(W * H, dtype=np.int32)
    o = oracle.render(sc, cam, env, pix, shade=False)
    OCH = {n: i for i, n in enumerate(oracle.CHANNELS)}
    Lr, gW = OR.opacity_loss(o["ch"][:, OCH["W"]].reshape(H, W))
    print("opacity loss gpu", L, "oracle", Lr)
    assert abs(L - Lr) <= 1e-5 * Lr
    g_ch = np.zeros((W * H, oracle.NDIFF))
    g_ch[:, OCH["W"]] = 1.5 * gW.reshape(-1)
    np.testing.assert_allclose(dg[N.CH["W"]].cpu().numpy(), g_ch[:, OCH["W"]], rtol=1e-6)
    d_s, _ = oracle.grad(sc, cam, env, pix, 0, 0, None, g_ch, shade=False)
    d_surf = torch.zeros((sc.n, 17), device="cuda")
    tr.backward(cam, g, 0, 1, 0, dL_dgbuf=dg, d_surfel=d_surf)
    tr.sync()
    gs = d_surf.cpu().numpy().astype(np.float64)
    for name, (a, b) in dict(mu=(0, 3), tu=(3, 6), tv=(6, 9), scale=(9, 11), opacity=(11, 12)).items():
        rel = np.linalg.norm(gs[:, a:b] - d_s[:, a:b]) / np.linalg.norm(d_s[:, a:b])
        print("opacity adjoint", name, rel)
        assert rel <= 1e-3, name
