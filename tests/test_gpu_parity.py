"""CUDA path against the FP64 oracle on the same seeded inputs (through the C ABI).

G-buffer: 1e-4 absolute per channel on every pixel whose primary ray the
oracle does not flag as sitting on a discontinuity; hit counts identical
there.  Shading (Eq. 11): per shading sample, the sample's share
(1 - T) / spp * c_s of its pixel within 1e-4 * max(1, |share|) on every
sample the oracle does not flag, and each pixel with its flagged samples
removed on both sides within 1e-4 * max(1, |L|) (unclamped) and 1e-4 on
[0, 1]; the flagged fractions (pixels by their primary ray, samples) are
printed and stay below 1 %.
"""

import numpy as np
import pytest

import oracle
from synthetic import scenes as S
from tests._helpers import (OCH, assert_shading, compare_gbuf, compare_samples, flagged, gbuf_at, gpu_shaded,
                            gpu_tracer, sample_flags)

pytestmark = pytest.mark.gpu
TOL = 1e-4


def test_philox_matches_known_answers_and_oracle():
    import torch
    tr, _ = gpu_tracer(S.scene_c1(), [S.env_uniform(1.0, 8, 16)])
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = [0, 0, 0, 0]
    for k0, k1 in [(0, 0), (0xa4093822, 0x299f31d0), (12345, 678)]:
        g = tr.philox(torch.as_tensor(ctr.view(np.int32), device="cuda"), k0, k1).cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(g, oracle.philox(ctr, k0, k1))
    g = tr.philox(torch.as_tensor(np.zeros((1, 4), np.int32), device="cuda"), 0, 0).cpu().numpy().view(np.uint32)
    assert [hex(int(v)) for v in g[0]] == ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]


@pytest.mark.parametrize("env", [S.env_sky_sun(0), S.env_smooth(1, 64, 128)])
def test_env_tables_match_oracle(env):
    tr, _ = gpu_tracer(S.scene_c1(), [env])
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in tr.env_tables(0).items()}
    o = oracle.env_tables(env)
    # both sides sum in FP64 in the same order; the FP32 tables must agree exactly
    for k in ["cdf_row", "cdf_col"]:
        np.testing.assert_array_equal(g[k], o[k].astype(np.float32).astype(np.float64))
    for k in ["pmf_row", "pmf_col"]:
        np.testing.assert_allclose(g[k], o[k], rtol=1.2e-7, atol=0)


def _c1_inputs():
    return S.scene_c1(0), S.camera_c1(), S.env_uniform(1.0)


def test_c1_primary_gbuffer_parity():
    sc, cam, env = _c1_inputs()
    tr, _ = gpu_tracer(sc, [env])
    g = tr.trace_primary(cam, 0)
    tr.sync()
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    o = oracle.render(sc, cam, env, pix, shade=False)
    gg = gbuf_at(g, pix)
    flag = flagged(o["margins"])
    ok = ~flag
    assert flag.mean() < 0.01
    assert (o["ch"][:, OCH["hits"]] > 0).sum() > 400
    np.testing.assert_array_equal(gg[ok, 18], o["ch"][ok, OCH["hits"]])
    errs = compare_gbuf(gg, o["ch"], ok)
    print("C1 gbuf max errors:", errs, "flagged:", int(flag.sum()))
    assert max(errs.values()) <= TOL, errs


@pytest.mark.parametrize("params", [dict(), dict(sampling_mode=1), dict(sampling_mode=2), dict(brdf_mode=1),
                                    dict(sampler=1)])
def test_c1_shaded_parity(params):
    sc, cam, _ = _c1_inputs()
    env = S.env_sky_sun(3)
    tr, _ = gpu_tracer(sc, [env], **params)
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    _, _, gg, terms, rgb = gpu_shaded(tr, cam, 0, 8, 77, pix)
    o = oracle.render(sc, cam, env, pix, spp=8, seed=77, params=params)
    r = compare_samples(o, terms, gg[:, 0], rgb, 8)
    print(params, "C1 shaded:", r)
    assert_shading(r)


def test_c2_one_bounce_parity_on_pixel_subset():
    """200k-surfel room, 800x800, 16 spp: full GPU frame, oracle on 4,096 seeded pixels."""
    sc, cam, env = S.scene_c2(0), S.camera_c2(), S.env_sky_sun(0)
    tr, _ = gpu_tracer(sc, [env])
    pix = S.pixel_subset(cam.width, cam.height, 4096, seed=5)
    _, _, gg, terms, rgb = gpu_shaded(tr, cam, 0, 16, 1234, pix)
    o = oracle.render(sc, cam, env, pix, spp=16, seed=1234)
    flag_p = flagged(o["margins"])
    errs = compare_gbuf(gg, o["ch"], ~flag_p)
    r = compare_samples(o, terms, gg[:, 0], rgb, 16)
    print("C2 gbuf errs", errs, "shading", r)
    assert (o["ch"][:, OCH["hits"]] > 0).mean() > 0.9
    np.testing.assert_array_equal(gg[~flag_p, 18], o["ch"][~flag_p, OCH["hits"]])
    assert max(errs.values()) <= TOL
    assert_shading(r)
    # The record's residual planes carry the composite below FP32: x + x_lo,
    # n + n_lo and r + r_lo stay within ~1e-9 of the oracle's FP64 values at
    # the median pixel (the FP32 values alone: ~3e-8, one rounding).  The
    # tail (~1e-7) is set by the FP32 opacities and transmittances of the
    # weights where a pixel blends surfaces a distance apart.
    ok = ~flag_p & (o["ch"][:, OCH["hits"]] > 0)
    for ch, lo, oc, k in [(3, 25, OCH["x0"], 3), (6, 28, OCH["n0"], 3), (13, 31, OCH["r"], 1)]:
        err_hi = np.abs(gg[ok, ch:ch + k] - o["ch"][ok, oc:oc + k]).max(1)
        err = np.abs(gg[ok, ch:ch + k] + gg[ok, lo:lo + k] - o["ch"][ok, oc:oc + k]).max(1)
        print("C2 record residual", ch, "median", np.median(err), "q99", np.quantile(err, 0.99),
              "FP32 value alone median", np.median(err_hi))
        assert np.median(err) <= 1e-8
        assert np.quantile(err, 0.99) <= 2e-7
        assert np.median(err) <= np.median(err_hi)


def test_c4_layout_parity_on_pixel_subset():
    """Multi-state relighting scene: 1M surfels (shell + 12 objects), 1024x1024,
    64 spp, the third environment state, after a layout that moves three
    objects (rotation about +y, x/z shift; BLAS refit on the GPU, Eq. 2 in the
    oracle): the moved surfels equal the oracle's bit for bit, the G-buffer
    and every unflagged shading sample match it on 256 seeded pixels, and the
    adjoint of a loss on the pixels without a flagged sample matches the
    oracle's gradient."""
    import torch
    sc, cam = S.scene_c4(0), S.camera_c4()
    envs = [S.env_sky_sun(k) for k in range(3)]
    tr, st = gpu_tracer(sc, envs)
    rng = np.random.default_rng(21)
    ref = sc
    for obj in rng.choice(np.arange(1, sc.n_objects), 3, replace=False):
        lo, hi = sc.object_offsets[obj], sc.object_offsets[obj + 1]
        R, t = S.rigid_motion(rng, sc.mu[lo:hi].mean(0))
        tr.refit(int(obj), R, t)
        ref = oracle.rigid(ref, int(obj), R, t)
    tr.sync()
    for k in ["mu", "tu", "tv"]:
        np.testing.assert_array_equal(getattr(st, k).cpu().numpy(), getattr(ref, k))
    spp, seed, env_id = 64, 77, 2
    pix = S.pixel_subset(cam.width, cam.height, 256, seed=9)
    g, samples, gg, terms, rgb = gpu_shaded(tr, cam, env_id, spp, seed, pix)
    o = oracle.render(ref, cam, envs[env_id], pix, spp=spp, seed=seed)
    flag_p = flagged(o["margins"])
    errs = compare_gbuf(gg, o["ch"], ~flag_p)
    r = compare_samples(o, terms, gg[:, 0], rgb, spp)
    print("C4 gbuf errs", errs, "shading", r)
    assert max(errs.values()) <= TOL
    # The shell of this scene holds 4x the surfels per unit area of the
    # 200k room's, so about twice C2's fraction of shading rays pass within
    # the ray-shift allowance of a support edge or a depth tie (~0.8 %).
    assert_shading(r)
    # adjoint of a loss on the sampled pixels none of whose decisions is flagged
    ok = ~(flag_p | sample_flags(o).any(1))
    print("C4 gradient pixels", int(ok.sum()), "of", len(pix))
    assert ok.sum() >= 128  # flags cluster in pixels: well over half of them have none
    g_rgb = rng.normal(size=(len(pix), 3)) * ok[:, None]
    d_s, d_e = oracle.grad(ref, cam, envs[env_id], pix, spp, seed, g_rgb)
    full = torch.zeros((cam.height * cam.width, 3), device="cuda")
    full[torch.as_tensor(pix.astype(np.int64), device="cuda")] = torch.as_tensor(g_rgb, dtype=torch.float32,
                                                                                  device="cuda")
    d_surf = torch.zeros((sc.n, 17), device="cuda")
    d_env = torch.zeros((envs[env_id].height, envs[env_id].width, 3), device="cuda")
    tr.backward(cam, g, env_id, spp, seed, dL_drgb=full.contiguous(), d_surfel=d_surf, d_env=d_env,
                fwd_samples=samples)
    tr.sync()
    gs, ge = d_surf.cpu().numpy().astype(np.float64), d_env.cpu().numpy().astype(np.float64)
    groups = dict(mu=(0, 3), tu=(3, 6), tv=(6, 9), scale=(9, 11), opacity=(11, 12), albedo=(12, 15),
                  metallic=(15, 16), roughness=(16, 17))
    pairs = {k: (d_s[:, a:b], gs[:, a:b]) for k, (a, b) in groups.items()}
    pairs["env"] = (d_e, ge)
    for name, (ref_g, got) in pairs.items():
        rel = np.linalg.norm(got - ref_g) / np.linalg.norm(ref_g)
        print("C4 gradient", name, "L2-relative", rel)
        assert rel <= 1e-3, name


def test_refit_matches_rebuild_bitwise():
    """Refit keeps the topology; the hit sets, and so the G-buffer, equal a fresh build."""
    import torch
    sc, cam, env = S.scene_c2(0, per_face=3000, per_object=8000), S.camera_c2(200, 200), S.env_sky_sun(1)
    tr, st = gpu_tracer(sc, [env])
    rng = np.random.default_rng(4)
    for obj in [1, 3]:
        lo, hi = sc.object_offsets[obj], sc.object_offsets[obj + 1]
        R, t = S.rigid_motion(rng, sc.mu[lo:hi].mean(0))
        tr.refit(obj, R, t)
    g1 = tr.trace_primary(cam, 0).clone()
    tr.sync()
    moved = st.mu.cpu().numpy()
    ref = sc.copy()
    ref.mu, ref.tu, ref.tv = moved, st.tu.cpu().numpy(), st.tv.cpu().numpy()
    tr2, _ = gpu_tracer(ref, [env])
    g2 = tr2.trace_primary(cam, 0)
    tr2.sync()
    assert torch.equal(g1, g2)
    # and the moved object really moved
    assert not np.allclose(moved[sc.object_offsets[1]:sc.object_offsets[2]], sc.mu[sc.object_offsets[1]:sc.object_offsets[2]])


def test_bvh_boxes_nest_and_cover_every_leaf():
    sc = S.scene_c2(0, per_face=2000, per_object=5000)
    tr, _ = gpu_tracer(sc, [S.env_uniform(1.0, 8, 16)])
    for obj in range(sc.n_objects):
        nodes, root = tr.bvh_nodes(obj)
        n_leaves = sc.object_offsets[obj + 1] - sc.object_offsets[obj]
        assert len(nodes) == n_leaves - 1 and root == 0
        seen = np.zeros(n_leaves, int)
        # child codes: >= 0 internal, < 0 leaf ~code
        codes = nodes[:, 12:14].copy().view(np.int32)
        box = lambda n, side: (nodes[n, 0:3], nodes[n, 3:6]) if side == 0 else (nodes[n, 6:9], nodes[n, 9:12])
        stack = [0]
        while stack:
            n = stack.pop()
            for side in (0, 1):
                c = int(codes[n, side])
                if c >= 0:
                    lo, hi = box(n, side)
                    for cs in (0, 1):
                        clo, chi = box(c, cs)
                        assert np.all(clo >= lo) and np.all(chi <= hi)
                    stack.append(c)
                else:
                    seen[~c] += 1
        assert np.all(seen == 1)


def test_wide_bvh_covers_every_leaf_once_and_nests():
    """The wide BVH collapsed from the binary one: every surfel in exactly one
    leaf slot, child slot boxes inside their parent slot's box, leaf slots of
    at most WIDE surfels, node count within the per-object capacity."""
    sc = S.scene_c2(0, per_face=2000, per_object=5000)
    tr, _ = gpu_tracer(sc, [S.env_uniform(1.0, 8, 16)])
    nodes_b = {}
    for obj in range(sc.n_objects):
        slots, root, rcount = tr.bvh_wide(obj)
        n_leaves = sc.object_offsets[obj + 1] - sc.object_offsets[obj]
        wide = slots.shape[1]
        seen = np.zeros(n_leaves, int)
        if root < 0:
            assert n_leaves <= wide and rcount == n_leaves
            continue
        codes = slots[:, :, 3].copy().view(np.int32)
        counts = slots[:, :, 7].copy().view(np.int32)
        visited = set()
        stack = [0]
        while stack:
            n = stack.pop()
            assert n not in visited and n < len(slots)
            visited.add(n)
            for c in range(wide):
                code = int(codes[n, c])
                if code == np.iinfo(np.int32).min:
                    continue
                lo, hi = slots[n, c, 0:3], slots[n, c, 4:7]
                assert np.all(lo <= hi)
                if code >= 0:
                    clive = codes[code] != np.iinfo(np.int32).min
                    assert clive.sum() >= 2
                    # compressed boxes are rounded outward per node (FP16 offsets from the node
                    # centre): a child may stick out of its parent's slot by one FP16 step
                    tol = 2.0 ** -10 * (hi - lo) + 1e-6
                    assert np.all(slots[code, clive, 0:3] >= lo - tol) and np.all(slots[code, clive, 4:7] <= hi + tol)
                    stack.append(code)
                else:
                    first, cnt = ~code, int(counts[n, c])
                    assert 1 <= cnt <= wide
                    seen[first:first + cnt] += 1
        assert np.all(seen == 1), obj
        assert len(visited) <= len(slots)


@pytest.mark.parametrize("params", [dict(), dict(sampler=1)])
def test_c3_gradient_parity(params):
    """Adjoint vs the oracle's reverse-mode gradient (1e-3 relative), 512 surfels, 32x32, 4 spp."""
    import torch
    from paper_2608_29269_b300 import _native as N
    full = S.scene_c2(0)
    cam = S.camera_c2(32, 32)
    sc = S.scene_c3_subset(full, cam, 512, seed=0)
    env = S.env_sky_sun(0)
    tr, st = gpu_tracer(sc, [env], **params)
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    o = oracle.render(sc, cam, env, pix, spp=4, seed=3, params=params)
    ok = ~(flagged(o["margins"], FLAG_GRAD) | sample_flags(o).any(1))
    rng = np.random.default_rng(8)
    g_rgb = rng.normal(size=(cam.n_pixels, 3)) * ok[:, None]
    g_ch = rng.normal(size=(cam.n_pixels, 17)) * 0.2 * ok[:, None]
    d_s, d_e = oracle.grad(sc, cam, env, pix, 4, 3, g_rgb, g_ch, params=params)
    g = tr.trace_primary(cam, 0)
    samples = tr.alloc_samples(cam, 4)
    tr.shade(cam, g, 0, spp=4, seed=3, samples=samples)
    gg = torch.zeros((N.LF_GBUF_CHANNELS, cam.height * cam.width), device="cuda")
    gg[:17] = torch.as_tensor(g_ch.T, dtype=torch.float32, device="cuda")
    d_surf = torch.zeros((sc.n, 17), device="cuda")
    d_env = torch.zeros((env.height, env.width, 3), device="cuda")
    tr.backward(cam, g, 0, 4, 3, dL_drgb=torch.as_tensor(g_rgb, dtype=torch.float32, device="cuda").contiguous(),
                dL_dgbuf=gg.contiguous(), d_surfel=d_surf, d_env=d_env, fwd_samples=samples)
    tr.sync()
    gs, ge = d_surf.cpu().numpy().astype(np.float64), d_env.cpu().numpy().astype(np.float64)
    # the replayed adjoint (no forward buffer) gives the same gradients
    d_surf2, d_env2 = torch.zeros_like(d_surf), torch.zeros_like(d_env)
    tr.backward(cam, g, 0, 4, 3, dL_drgb=torch.as_tensor(g_rgb, dtype=torch.float32, device="cuda").contiguous(),
                dL_dgbuf=gg.contiguous(), d_surfel=d_surf2, d_env=d_env2)
    tr.sync()
    np.testing.assert_allclose(d_surf2.cpu().numpy(), gs, rtol=1e-5, atol=1e-6 * np.abs(gs).max())
    np.testing.assert_allclose(d_env2.cpu().numpy(), ge, rtol=1e-5, atol=1e-6 * np.abs(ge).max())
    # Criterion: per attribute group the L2-relative error is at most 1e-3, and
    # element-wise |g - g_ref| <= 1e-3 |g_ref| + 1e-4 max|g_ref| (the floor covers
    # FP32 cancellation when large per-pixel contributions sum to a small value).
    report, worst = {}, {}
    groups = dict(mu=(0, 3), tu=(3, 6), tv=(6, 9), scale=(9, 11), opacity=(11, 12), albedo=(12, 15),
                  metallic=(15, 16), roughness=(16, 17))
    pairs = {k: (d_s[:, a:b], gs[:, a:b]) for k, (a, b) in groups.items()}
    pairs["env"] = (d_e, ge)
    for name, (ref, got) in pairs.items():
        report[name] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        worst[name] = float((np.abs(got - ref) / (1e-3 * np.abs(ref) + 1e-4 * np.abs(ref).max())).max())
    print("gradient L2-relative errors:", report, "element-wise (<=1):", worst,
          "nonzero surfels", int((np.abs(d_s).sum(1) > 0).sum()))
    assert (np.abs(d_s).sum(1) > 0).sum() > 50
    assert max(report.values()) <= 1e-3, report
    assert max(worst.values()) <= 1.0, worst


FLAG_GRAD = dict(support=1e-6, alpha=1e-6, tmin=1e-5, tie=1e-9, stop=2e-5, cos=2e-6, frame=2e-6, cap=1e-5)


def test_counters_and_kernel_timing_are_consistent():
    """Per-kernel counter slots add up to the rays the shading reports, and
    the per-kernel event timings are positive and inside the call's span."""
    import torch
    sc, cam, env = _c1_inputs()
    tr, _ = gpu_tracer(sc, [env])
    cnt = torch.zeros(20, dtype=torch.int64, device="cuda")
    rays = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        tr.set_counters(torch.zeros(4, dtype=torch.int64, device="cuda"))
    tr.set_counters(cnt)
    tr.profile(True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tr.sync()
    t0.record()
    g = tr.trace_primary(cam, 0)
    samples = tr.alloc_samples(cam, 4)
    tr.shade(cam, g, 0, spp=4, seed=5, ray_count=rays, samples=samples)
    assert tr.profile_read()[6:] == [0.0, 0.0]  # no backward profiled yet
    d_s = torch.zeros((sc.n, 17), device="cuda")
    tr.backward(cam, g, 0, 4, 5, dL_drgb=torch.ones((cam.height, cam.width, 3), device="cuda"), d_surfel=d_s,
                fwd_samples=samples)
    tr.sync()
    t1.record()
    torch.cuda.synchronize()
    ms = tr.profile_read()
    tr.profile(False)
    tr.set_counters(None)
    c = cnt.cpu().numpy().reshape(5, 4)
    hits = int((g[18] > 0).sum().item())
    assert c[0, 3] == cam.width * cam.height
    # the adjoint re-traverses every pixel with a hit and scatters each composited hit once
    assert c[4, 3] == hits and c[4, 2] == c[0, 2] and c[4, 0] > 0 and c[4, 1] > 0
    assert c[1, 3] + c[2, 3] + c[3, 3] == int(rays.item())
    for k in range(4):
        if c[k, 3] > 0:
            assert c[k, 0] > 0 and c[k, 1] > 0
    assert c[0, 2] > 0 and c[2, 2] >= 0 and c[1, 2] == 0 and c[3, 2] == 0
    assert len(ms) == 8 and all(v > 0 for v in ms)
    assert sum(ms) <= t0.elapsed_time(t1) * 1.05 + 0.05
