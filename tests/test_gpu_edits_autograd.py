"""The served edits of Sec. 3.4.2 (material edits, an environment swap, a
rigid move) and the torch.autograd.Function behind the hand-written adjoint
(Sec. 3.3 path replay), checked element by element against the FP64 oracle.

An oracle-side material edit is a plain write into the scene's arrays, an
environment swap renders with the other map, a move is Eq. 2 (oracle.rigid).
Radiance is compared per shading sample where the sample terms are
available (lf_shade_sample_terms) and per pixel for the server's frames
(pixels with a flagged decision left out and counted); gradients at the
1e-3 relative bound of the parity tests.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from synthetic import scenes as S
from tests._helpers import FLAG, assert_shading, compare_samples, flagged, gpu_tracer, sample_flags

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _room():
    return S.scene_c2(0, per_face=3000, per_object=8000)


def _envs():
    return [S.env_sky_sun(i, 64, 128) for i in range(3)]


def _material(scene, obj, albedo=None, metallic=None, roughness=None):
    """Oracle side of lf_material_set: overwrite the object's arrays."""
    out = scene.copy()
    lo, hi = int(scene.object_offsets[obj]), int(scene.object_offsets[obj + 1])
    if albedo is not None:
        out.albedo[lo:hi] = np.asarray(albedo, np.float32)
    if metallic is not None:
        out.metallic[lo:hi] = np.float32(metallic)
    if roughness is not None:
        out.roughness[lo:hi] = np.float32(roughness)
    return out


def test_material_edit_and_env_swap_match_oracle_per_sample():
    sc, envs = _room(), _envs()
    tr, st = gpu_tracer(sc, envs)
    tr.set_material(2, (0.9, 0.2, 0.1), 0.8, 0.3)
    tr.set_material(3, None, -1.0, 0.6)  # roughness only
    tr.set_material(4, (0.05, 0.5, 0.95), 0.0, -1.0)
    ref = _material(_material(_material(sc, 2, (0.9, 0.2, 0.1), 0.8, 0.3), 3, roughness=0.6), 4, (0.05, 0.5, 0.95),
                    0.0)
    tr.sync()
    for k in ["albedo", "metallic", "roughness"]:  # the edit wrote the caller's arrays
        np.testing.assert_array_equal(getattr(st, k).cpu().numpy(), getattr(ref, k))
    cam = S.Camera((0.0, -0.5, 1.8), (0.0, -1.5, 0.0), (0.0, 1.0, 0.0), 60.0, 48, 48)
    spp, seed = 4, 21
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    for env_id in (2, 1):  # the swap: the same edited scene under another environment
        g = tr.trace_primary(cam, env_id)
        samples = tr.alloc_samples(cam, spp)
        rgb = tr.shade(cam, g, env_id, spp=spp, seed=seed, samples=samples)
        terms = tr.sample_terms(cam, g, env_id, spp, samples)
        tr.sync()
        o = oracle.render(ref, cam, envs[env_id], pix, spp=spp, seed=seed)
        r = compare_samples(o, terms.cpu().numpy(), g[0].reshape(-1).cpu().numpy(),
                            rgb.reshape(-1, 3).cpu().numpy(), spp)
        print("material edit, env", env_id, r)
        assert_shading(r)


def test_served_edits_match_oracle():
    """Each served frame equals the oracle's render of the scene state right
    after its own edit (edits apply in submission order)."""
    from paper_2608_29269_b300.serve import Server, run_served
    from synthetic.requests import Request
    sc, envs = _room(), _envs()
    tr, st = gpu_tracer(sc, envs)
    cam = lambda res: S.Camera((0.0, -0.5, 1.8), (0.0, -1.5, 0.0), (0.0, 1.0, 0.0), 60.0, res, res)
    lo, hi = sc.object_offsets[1], sc.object_offsets[2]
    R, t = S.rigid_motion(np.random.default_rng(5), sc.mu[lo:hi].mean(0), max_shift=0.2)
    edits = [dict(kind="material", object=2, albedo=np.array([0.9, 0.3, 0.2], np.float32), metallic=0.7,
                  roughness=0.25),
             dict(kind="env", env=1),
             dict(kind="move", object=1, R=R, t=t),
             dict(kind="material", object=3, roughness=0.8),
             dict(kind="env", env=2)]
    reqs = [Request(0.0, e, cam(res), spp, seed) for e, res, spp, seed in
            zip(edits, (40, 32, 48, 40, 32), (3, 4, 2, 4, 3), (1, 2, 3, 4, 5))]
    srv = Server(tr, budget_bytes=2 << 30, max_slots=4, n_streams=2, batch_window_us=20_000)
    out = run_served(srv, reqs, keep_frames=True)
    srv.close()
    state, env_id = sc, 0
    for rq, res in zip(reqs, out):
        e = rq.edit
        if e["kind"] == "material":
            state = _material(state, e["object"], e.get("albedo"), e.get("metallic"), e.get("roughness"))
        elif e["kind"] == "move":
            state = oracle.rigid(state, e["object"], e["R"], e["t"])
        else:
            env_id = e["env"]
        assert res["status"] == 0, res["status"]
        pix = np.arange(rq.cam.n_pixels, dtype=np.int32)
        o = oracle.render(state, rq.cam, envs[env_id], pix, spp=rq.spp, seed=rq.seed)
        bad = sample_flags(o).any(1)
        frame = res["frame"].reshape(-1, 3).astype(np.float64)
        rel = (np.abs(frame - o["rgb"]) / np.maximum(1.0, np.abs(o["rgb"])))[~bad]
        print(e["kind"], "frame", rq.cam.width, "flagged pixels", bad.mean(), "max rel", rel.max())
        assert bad.mean() < 0.05 and rel.max() <= TOL


def test_autograd_function_matches_oracle_gradient():
    """render() / SurfelRender.apply with requires_grad tensors and
    loss.backward(): the .grad of every surfel tensor and of the environment
    against the oracle's reverse-mode gradient under the same freeze."""
    import torch
    from paper_2608_29269_b300 import SceneTensors, Tracer
    from paper_2608_29269_b300.build import build
    from paper_2608_29269_b300.render import render
    build()
    full = S.scene_c2(0)
    cam = S.camera_c2(32, 32)
    sc = S.scene_c3_subset(full, cam, 512, seed=0)
    env = S.env_sky_sun(0)
    spp, seed = 4, 3
    tr = Tracer()
    st = SceneTensors.from_numpy(sc)
    for t in st.tensors():
        t.requires_grad_(True)
    tr.build(st)
    env_t = torch.as_tensor(env.rgb, device="cuda").contiguous().requires_grad_(True)
    tr.set_env(0, env_t)
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    o = oracle.render(sc, cam, env, pix, spp=spp, seed=seed)
    ok = ~(flagged(o["margins"], FLAG) | sample_flags(o).any(1))
    assert ok.mean() > 0.9
    w = np.random.default_rng(8).normal(size=(cam.n_pixels, 3)) * ok[:, None]
    rgb, gbuf = render(tr, cam, 0, spp, seed)
    loss = (rgb.reshape(-1, 3) * torch.as_tensor(w, dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    tr.sync()
    d_s, d_e = oracle.grad(sc, cam, env, pix, spp, seed, w)
    got = {k: getattr(st, k).grad.detach().reshape(sc.n, -1).cpu().numpy().astype(np.float64)
           for k in ["mu", "tu", "tv", "scale", "opacity", "albedo", "metallic", "roughness"]}
    groups = dict(mu=(0, 3), tu=(3, 6), tv=(6, 9), scale=(9, 11), opacity=(11, 12), albedo=(12, 15),
                  metallic=(15, 16), roughness=(16, 17))
    pairs = {k: (d_s[:, a:b], got[k]) for k, (a, b) in groups.items()}
    pairs["env"] = (d_e, env_t.grad.detach().cpu().numpy().astype(np.float64))
    for name, (ref, g) in pairs.items():
        rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        worst = (np.abs(g - ref) / (1e-3 * np.abs(ref) + 1e-4 * np.abs(ref).max())).max()
        print("autograd", name, "L2-relative", rel, "element-wise", worst)
        assert rel <= 1e-3 and worst <= 1.0, name
