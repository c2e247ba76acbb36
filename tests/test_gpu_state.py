"""Cross-state supervision (Sec. 3.2, Eq. 2) through the C ABI against the oracle:
state assembly and its adjoint bit for bit, and the gradient of a two-state
loss with respect to the shared canonical parameters."""
import numpy as np
import pytest

import oracle
from synthetic import scenes as S
from tests._helpers import sample_flags, flagged, gpu_tracer

pytestmark = pytest.mark.gpu

FLAG_GRAD = dict(support=1e-6, alpha=1e-6, tmin=1e-5, tie=1e-9, stop=2e-5, cos=2e-6, frame=2e-6, cap=1e-5)


def _state(rng, sc, max_shift=0.15):
    Rs, ts = [], []
    for o in range(1, sc.n_objects):
        lo, hi = sc.object_offsets[o], sc.object_offsets[o + 1]
        R, t = S.rigid_motion(rng, sc.mu[lo:hi].mean(0) if hi > lo else np.zeros(3), max_shift=max_shift)
        Rs.append(R)
        ts.append(t)
    return np.stack(Rs), np.stack(ts)


def _canonical_tensors(sc, share_attributes):
    """Canonical tensors, and the world scene the tracer is built on: its own
    centres and axes, and either its own or the canonical's other arrays."""
    import torch
    from paper_2608_29269_b300 import SceneTensors
    can = SceneTensors.from_numpy(sc)
    world = SceneTensors.from_numpy(sc)
    if share_attributes:
        for k in ["scale", "opacity", "albedo", "metallic", "roughness"]:
            setattr(world, k, getattr(can, k))
    else:
        for k in ["scale", "opacity", "albedo", "metallic", "roughness"]:
            getattr(world, k).zero_()
    return can, world


@pytest.mark.parametrize("share_attributes", [False, True])
def test_state_assembly_and_pullback_match_oracle_bitwise(share_attributes):
    import torch
    from paper_2608_29269_b300 import Tracer
    sc = S.scene_c2(0, per_face=2000, per_object=5000)
    cam, env = S.camera_c2(160, 160), S.env_sky_sun(0)
    can, world = _canonical_tensors(sc, share_attributes)
    tr = Tracer()
    tr.build(world)
    tr.set_env(0, torch.as_tensor(env.rgb, device="cuda"))
    rng = np.random.default_rng(21)
    for _ in range(2):  # two states in a row: the second starts from the first's world
        R, t = _state(rng, sc, max_shift=0.5)
        tr.assemble_state(can, R, t)
        tr.sync()
        ref = oracle.assemble_state(sc, R, t)
        for k in ["mu", "tu", "tv", "scale", "opacity", "albedo", "metallic", "roughness"]:
            np.testing.assert_array_equal(getattr(world, k).cpu().numpy(), getattr(ref, k), err_msg=k)
        # the refitted BVH traces exactly what a fresh build of the state traces
        g1 = tr.trace_primary(cam, 0).clone()
        tr2, _ = gpu_tracer(ref, [env])
        g2 = tr2.trace_primary(cam, 0)
        tr2.sync()
        assert torch.equal(g1, g2)
        # the adjoint, into a non-zero accumulator
        d_w = torch.randn((sc.n, 17), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
        acc0 = torch.randn((sc.n, 17), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
        acc = acc0.clone()
        tr.state_pullback(R, d_w, acc)
        tr.sync()
        want = oracle.state_pullback(sc.object_offsets, R, d_w.cpu().numpy()).astype(np.float32)
        np.testing.assert_array_equal(acc.cpu().numpy(), acc0.cpu().numpy() + want)  # one FP32 add each
        # the canonical arrays are left as they were
        np.testing.assert_array_equal(can.mu.cpu().numpy(), sc.mu)


def test_state_calls_reject_bad_arguments():
    import torch
    from paper_2608_29269_b300 import Tracer
    from paper_2608_29269_b300._native import LightFuseError
    sc = S.scene_c2(0, per_face=200, per_object=400)
    can, world = _canonical_tensors(sc, False)
    tr = Tracer()
    R, t = _state(np.random.default_rng(1), sc)
    with pytest.raises(LightFuseError, match="no BVH"):  # nothing built yet
        tr.check(tr.lib.lf_state_pullback(tr.ctx, None, None, None))
    tr.build(world)
    with pytest.raises(ValueError):
        tr.assemble_state(can, R[:-1], t[:-1])
    bad = R.copy()
    bad[0] *= 2.0
    with pytest.raises(LightFuseError, match="rigid"):
        tr.assemble_state(can, bad, t)
    with pytest.raises(LightFuseError, match="alias"):
        tr.assemble_state(world, R, t)
    g = torch.zeros((sc.n, 17), device="cuda")
    with pytest.raises(LightFuseError, match="overlap"):
        tr.state_pullback(R, g, g)


def test_cross_state_gradient_parity():
    """Two states of one canonical scene, rendered and differentiated through
    lf_state_assemble / lf_trace_backward / lf_state_pullback, against the
    oracle's per-state reverse-mode gradients carried back through Eq. 2
    (same criterion as the single-state gradient parity)."""
    import torch
    from paper_2608_29269_b300 import Tracer, render_state
    full = S.scene_c2(0)
    cam = S.camera_c2(32, 32)
    sc = S.scene_c3_subset(full, cam, 512, seed=0, keep_objects=True)
    assert sc.n_objects >= 3
    env = S.env_sky_sun(0)
    can, world = _canonical_tensors(sc, False)
    for k in can.tensors():
        k.requires_grad_(True)
    tr = Tracer()
    tr.build(world)
    env_t = torch.as_tensor(env.rgb, device="cuda").requires_grad_(True)
    tr.set_env(0, env_t.detach())
    tr.envs[0] = env_t
    rng = np.random.default_rng(31)
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    spp, seeds = 4, [3, 4]
    states = [_state(rng, sc) for _ in seeds]
    d_ref = np.zeros((sc.n, 17))
    e_ref = np.zeros(env.rgb.shape)
    loss = 0.0
    for (R, t), seed in zip(states, seeds):
        ws = oracle.assemble_state(sc, R, t)
        o = oracle.render(ws, cam, env, pix, spp=spp, seed=seed)
        ok = ~(flagged(o["margins"], FLAG_GRAD) | sample_flags(o).any(1))
        g_rgb = rng.normal(size=(cam.n_pixels, 3)) * ok[:, None]
        d_s, d_e = oracle.grad(ws, cam, env, pix, spp, seed, g_rgb, np.zeros((cam.n_pixels, 17)))
        d_ref += oracle.state_pullback(sc.object_offsets, R, d_s)
        e_ref += d_e
        rgb, _ = render_state(tr, can, R, t, cam, 0, spp, seed)
        loss = loss + (rgb.reshape(-1, 3) * torch.as_tensor(g_rgb, dtype=torch.float32, device="cuda")).sum()
    loss.backward()  # both states' adjoints run after the second assembly
    got = np.concatenate([k.grad.reshape(sc.n, -1).cpu().numpy() for k in can.tensors()], axis=1).astype(np.float64)
    ge = env_t.grad.cpu().numpy().astype(np.float64)
    groups = dict(mu=(0, 3), tu=(3, 6), tv=(6, 9), scale=(9, 11), opacity=(11, 12), albedo=(12, 15),
                  metallic=(15, 16), roughness=(16, 17))
    pairs = {k: (d_ref[:, a:b], got[:, a:b]) for k, (a, b) in groups.items()}
    pairs["env"] = (e_ref, ge)
    report, worst = {}, {}
    for name, (ref, g) in pairs.items():
        report[name] = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
        worst[name] = float((np.abs(g - ref) / (1e-3 * np.abs(ref) + 1e-4 * np.abs(ref).max())).max())
    print("cross-state gradient L2-relative errors:", report, "element-wise (<=1):", worst)
    moved = slice(int(sc.object_offsets[1]), sc.n)
    assert (np.abs(d_ref[moved]).sum(1) > 0).sum() > 50
    assert max(report.values()) <= 1e-3, report
    assert max(worst.values()) <= 1.0, worst
