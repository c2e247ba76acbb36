"""Edge cases of the CUDA path against the oracle: ragged image sizes, an
empty scene, objects whose surfel counts straddle the wide-BVH leaf size,
the maximum number of objects, one and many samples per pixel, and surfels
seen edge-on (rays parallel to their planes)."""
import numpy as np
import pytest

import oracle
from synthetic import scenes as S
from tests._helpers import (OCH, assert_shading, compare_gbuf, compare_samples, flagged, gbuf_at, gpu_shaded,
                            gpu_tracer)

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _check(sc, cam, env, spp=4, seed=11, shade=True):
    """G-buffer on unflagged primary rays, then (shade) every unflagged
    shading sample and pixel, flagged samples under 1 % (the per-sample
    comparison of the parity tests)."""
    tr, _ = gpu_tracer(sc, [env])
    pix = np.arange(cam.width * cam.height, dtype=np.int32)
    if shade:
        g, _, gg, terms, rgb = gpu_shaded(tr, cam, 0, spp, seed, pix)
    else:
        g = tr.trace_primary(cam, 0)
        tr.sync()
        gg = gbuf_at(g, pix)
    o = oracle.render(sc, cam, env, pix, spp=spp if shade else 0, seed=seed, shade=shade)
    flag_p = flagged(o["margins"])
    errs = compare_gbuf(gg, o["ch"], ~flag_p)
    np.testing.assert_array_equal(gg[~flag_p, 18], o["ch"][~flag_p, OCH["hits"]])
    assert max(errs.values()) <= TOL, errs
    if shade:
        r = compare_samples(o, terms, gg[:, 0], rgb, spp)
        print(cam.width, cam.height, spp, r)
        assert_shading(r)
    return o


@pytest.mark.parametrize("wh", [(37, 23), (1, 1), (5, 64), (129, 3)])
def test_ragged_image_sizes(wh):
    sc = S.scene_c1(0)
    cam = S.Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 60.0, wh[0], wh[1])
    _check(sc, cam, S.env_sky_sun(2, 32, 64))


def test_empty_scene_shows_the_environment():
    e = np.zeros((0, 3), np.float32)
    sc = S.Scene(e, e, e, np.zeros((0, 2), np.float32), np.zeros(0, np.float32), e, np.zeros(0, np.float32),
                 np.zeros(0, np.float32), np.array([0, 0], np.int32))
    cam = S.Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 60.0, 16, 12)
    o = _check(sc, cam, S.env_sky_sun(1, 32, 64))
    assert np.all(o["ch"][:, OCH["hits"]] == 0) and np.all(o["ch"][:, OCH["T"]] == 1.0)


def test_objects_straddling_the_leaf_size_and_the_object_limit():
    from paper_2608_29269_b300 import _native as N
    base = S.scene_c1(0)
    # objects of 1, 2, 31, 32, 33, 100 surfels and the rest
    sizes = [1, 2, 31, 32, 33, 100]
    offs = np.concatenate([[0], np.cumsum(sizes), [base.n]]).astype(np.int32)
    sc = base.copy()
    sc.object_offsets = offs
    cam = S.camera_c1(48, 48)
    _check(sc, cam, S.env_uniform(1.0, 16, 32), shade=False)
    # the maximum number of objects: 64 (the instance table holds LF_MAX_OBJECTS)
    many = base.copy()
    many.object_offsets = np.linspace(0, base.n, N.LF_MAX_OBJECTS + 1).astype(np.int32)
    _check(many, cam, S.env_sky_sun(4, 32, 64))


@pytest.mark.parametrize("spp", [1, 64])
def test_one_and_many_samples_per_pixel(spp):
    _check(S.scene_c1(0), S.camera_c1(32, 32), S.env_sky_sun(5, 32, 64), spp=spp)


def test_surfels_seen_edge_on():
    """Surfels whose planes contain the view direction: rays parallel to a
    plane never hit it; those a little off-axis do."""
    rng = np.random.default_rng(3)
    n = 300
    mu = rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32)
    # planes spanned by x and z: normal along y, the camera looks along -z
    tu = np.tile([1.0, 0.0, 0.0], (n, 1)).astype(np.float32)
    tv = np.tile([0.0, 0.0, 1.0], (n, 1)).astype(np.float32)
    half = n // 2  # half of them tilted slightly out of the view plane
    ang = rng.uniform(0.01, 0.2, half)
    tv[:half] = np.stack([np.zeros(half), np.sin(ang), np.cos(ang)], -1).astype(np.float32)
    sc = S.Scene(mu, tu, tv, rng.uniform(0.05, 0.15, (n, 2)).astype(np.float32),
                 rng.uniform(0.3, 1.0, n).astype(np.float32), rng.uniform(0, 1, (n, 3)).astype(np.float32),
                 rng.uniform(0, 1, n).astype(np.float32), rng.uniform(0.1, 1, n).astype(np.float32),
                 np.array([0, n], np.int32))
    cam = S.Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 40.0, 40, 40)
    o = _check(sc, cam, S.env_sky_sun(6, 32, 64))
    assert (o["ch"][:, OCH["hits"]] > 0).sum() > 20
