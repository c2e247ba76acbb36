"""A scene restored from a checkpoint (BVH and environment tables rebuilt on
load) renders and differentiates like the scene that was saved."""
import numpy as np
import pytest

from synthetic import scenes as S

pytestmark = pytest.mark.gpu


def test_restored_scene_traces_and_shades_identically(tmp_path):
    import torch
    from paper_2608_29269_b300 import Tracer, SceneTensors, load_checkpoint, restore, save_checkpoint
    sc = S.scene_c2(0, per_face=2000, per_object=5000)
    cam = S.camera_c2(96, 96)
    tr = Tracer()
    st = SceneTensors.from_numpy(sc)
    tr.build(st)
    env = torch.as_tensor(S.env_sky_sun(2).rgb, device="cuda")
    tr.set_env(1, env)
    tr.refit(2, *S.rigid_motion(np.random.default_rng(3), sc.mu[sc.object_offsets[2]:sc.object_offsets[3]].mean(0)))
    g1 = tr.trace_primary(cam, 1).clone()
    rgb1 = tr.shade(cam, g1, 1, spp=8, seed=99).clone()
    d1, _ = tr.backward(cam, g1, 1, 8, 99, dL_drgb=torch.ones_like(rgb1))
    tr.sync()
    path = tmp_path / "ck.npz"
    save_checkpoint(path, st, envs={1: env}, params=tr.params, seed=99, spp=8)
    ck = load_checkpoint(path)
    tr2 = Tracer(**ck.params)
    restore(tr2, ck)
    g2 = tr2.trace_primary(cam, 1)
    rgb2 = tr2.shade(cam, g2, 1, spp=ck.spp, seed=ck.seed)
    d2, _ = tr2.backward(cam, g2, 1, ck.spp, ck.seed, dL_drgb=torch.ones_like(rgb2))
    tr2.sync()
    # the composites are sorted, so the G-buffer is the same bit for bit; the
    # rebuilt BVH groups the leaves differently, so shadow transmittance
    # products multiply in another order (rounding-level differences)
    assert torch.equal(g1, g2)
    np.testing.assert_allclose(rgb2.cpu().numpy(), rgb1.cpu().numpy(), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(d2.cpu().numpy(), d1.cpu().numpy(), rtol=1e-5, atol=1e-6 * d1.abs().max().item())
