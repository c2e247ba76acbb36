"""The oracle's reverse-mode gradient against FP64 central finite differences.

F(theta; frozen) is the rendered image with the path-replay data (sampled
directions, pdfs, MIS weights, visibilities, secondary records) frozen at
theta_0 (Sec. 3.3).  The finite difference re-renders with the perturbed
parameters while the frozen data still come from theta_0, so both sides
differentiate the same function.  A parameter whose perturbation changes a
discrete decision of the primary composite (hit set, order, stop index) or
crosses the 0.99 opacity cap is skipped.
"""
import numpy as np
import pytest

import oracle
from synthetic.scenes import Camera, Scene, env_smooth, quat_to_axes

CH = {n: i for i, n in enumerate(oracle.CHANNELS)}


def cluster_scene(n=24, seed=0):
    rng = np.random.default_rng(seed)
    mu = np.stack([rng.uniform(-0.25, 0.25, n), rng.uniform(-0.25, 0.25, n), rng.uniform(-0.3, 0.3, n)], 1)
    q = rng.normal(size=(n, 4))
    q[:, 0] += 2.5  # mostly facing the camera
    tu, tv = quat_to_axes(q)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    return Scene(f(mu), f(tu), f(tv), f(rng.uniform(0.06, 0.14, (n, 2))), f(rng.uniform(0.3, 0.95, n)),
                 f(rng.uniform(0.1, 0.9, (n, 3))), f(rng.uniform(0, 1, n)), f(rng.uniform(0.2, 0.9, n)),
                 np.array([0, n], np.int32))


FIELDS = [("mu", 3), ("tu", 3), ("tv", 3), ("scale", 2), ("opacity", 1), ("albedo", 3), ("metallic", 1),
          ("roughness", 1)]


def _param_ref(k):
    """Column k of the 17-wide gradient -> (field, component)."""
    for name, w in FIELDS:
        if k < w:
            return name, k
        k -= w
    raise IndexError


def _loss(out, g_rgb, g_ch):
    return float((out["rgb"] * g_rgb).sum() + (out["ch"][:, :17] * g_ch).sum())


@pytest.mark.parametrize("spp,params", [(2, {}), (2, dict(sampling_mode=1)), (1, dict(brdf_mode=1))])
def test_oracle_gradient_matches_central_differences(spp, params):
    sc = cluster_scene()
    cam = Camera((0, 0, 2.2), (0, 0, 0), (0, 1, 0), 22.0, 12, 12)
    env = env_smooth(7, 16, 32)
    pix = np.arange(cam.width * cam.height, dtype=np.int32)
    rng = np.random.default_rng(1)
    g_rgb = rng.normal(size=(len(pix), 3))
    g_ch = rng.normal(size=(len(pix), 17)) * 0.3
    seed = 9
    d_s, d_e = oracle.grad(sc, cam, env, pix, spp, seed, g_rgb, g_ch, params=params)
    base = oracle.render(sc, cam, env, pix, spp, seed, params=params)
    sig0 = base["ch"][:, CH["sig"]]
    hit_ids = np.unique(base["ch"][base["ch"][:, CH["hits"]] > 0, CH["id_stop"]]).astype(int)
    assert len(hit_ids) >= 5
    gscale = np.abs(d_s).max()
    checked = 0
    for sid in hit_ids[:8]:
        for k in range(17):
            name, comp = _param_ref(k)
            arr = getattr(sc, name)
            v0 = float(arr.reshape(sc.n, -1)[sid, comp])
            h = 2e-6 * max(1.0, abs(v0))
            vals, outs = [], []
            for sgn in (+1, -1):
                s2 = sc.copy()
                a2 = getattr(s2, name).reshape(s2.n, -1)
                a2[sid, comp] = np.float32(v0 + sgn * h)
                vals.append(float(a2[sid, comp]))
                outs.append(oracle.render(s2, cam, env, pix, spp, seed, params=params, scene0=sc))
            if any(np.any(o["ch"][:, CH["sig"]] != sig0) for o in outs):
                continue
            if np.any(np.minimum(outs[0]["margins"][:, 2], outs[1]["margins"][:, 2]) < 1e-5):
                continue
            fd = (_loss(outs[0], g_rgb, g_ch) - _loss(outs[1], g_rgb, g_ch)) / (vals[0] - vals[1])
            g = d_s[sid, k]
            assert abs(g - fd) <= 2e-5 * max(abs(fd), 1e-3 * gscale), (sid, name, comp, g, fd)
            checked += 1
    assert checked >= 60
    # environment texels (lookups are live, the sampling tables frozen)
    nz = np.argwhere(np.abs(d_e).sum(-1) > 0)
    pick = nz[np.random.default_rng(2).permutation(len(nz))[:12]]
    escale = np.abs(d_e).max()
    for (r, c) in pick:
        for ch in range(3):
            vals, losses = [], []
            for sgn in (+1, -1):
                e2 = env.rgb.copy()
                v0 = float(e2[r, c, ch])
                e2[r, c, ch] = np.float32(v0 + sgn * 1e-4)
                vals.append(float(e2[r, c, ch]))
                o = oracle.render(sc, cam, type(env)(e2), pix, spp, seed, params=params, env0=env)
                losses.append(_loss(o, g_rgb, g_ch))
            fd = (losses[0] - losses[1]) / (vals[0] - vals[1])
            assert abs(d_e[r, c, ch] - fd) <= 1e-6 * max(abs(fd), 1e-3 * escale) + 1e-9, (r, c, ch)
