"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than its own code: the
published Philox known-answer vectors, closed forms of Eq. 6-7 for hand-built
surfel configurations, an independent brute-force restatement of the
intersection (a 3x3 linear solve instead of the projection formula) and of
the compositing (explicit products instead of the running transmittance),
invariants (W = 1 - T, permutation invariance), white-furnace identities of
the estimator (Eq. 10-11), quadrature of the rendering integral, closed forms
of the GGX/Smith/Schlick BRDF and histogram tests of the samplers.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from synthetic.scenes import Camera, EnvMap, Scene, env_smooth, env_uniform, scene_c1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CH = {n: i for i, n in enumerate(oracle.CHANNELS)}
MG = {n: i for i, n in enumerate(oracle.MARGINS)}


def make_scene(surfels):
    """surfels: list of dicts with mu, tu, tv, s, o, a, m, r."""
    f = lambda k, d=None: np.array([np.asarray(s.get(k, d), np.float64) for s in surfels], np.float32)
    n = len(surfels)
    return Scene(f("mu"), f("tu"), f("tv"), f("s"), f("o"), f("a", (0.5, 0.5, 0.5)), f("m", 0.0), f("r", 0.5),
                 np.array([0, n], np.int32))


def disk(z=0.0, o=0.5, s=(0.1, 0.1), a=(0.2, 0.4, 0.6), m=0.0, r=0.5, flip=False, x=0.0, y=0.0):
    tu, tv = ((0, 1, 0), (1, 0, 0)) if flip else ((1, 0, 0), (0, 1, 0))
    return dict(mu=(x, y, z), tu=tu, tv=tv, s=s, o=o, a=a, m=m, r=r)


def trace1(scene, origin, direction, env=None, **params):
    env = env or env_uniform(0.7, 8, 16)
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    ch, mg = oracle.trace_rays(scene, env, np.asarray(origin, np.float64)[None], d[None], oracle.default_params(**params))
    return ch[0], mg[0]


# ---------------------------------------------------------------- Philox


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    for row in rows:
        v = [int(x, 16) for x in row]
        out = oracle.philox([v[0:4]], v[4], v[5])[0]
        assert [int(x) for x in out] == v[6:10]


def test_uniforms_are_24_bit_and_in_unit_interval():
    u = np.concatenate([oracle.uniforms(p, s, 12345) for p in range(50) for s in range(4)])
    assert np.all(u >= 0) and np.all(u < 1)
    assert np.all(np.round(u * 2 ** 24) == u * 2 ** 24)


# ---------------------------------------------------------------- Sobol sampler (variant of the paper's replayed Sobol samples)


def test_sobol_first_dimension_is_van_der_corput():
    i = np.arange(4096, dtype=np.uint32)
    rev = np.array([int(f"{x:032b}"[::-1], 2) for x in i], np.uint64)
    np.testing.assert_array_equal(oracle.sobol(i, 0).astype(np.uint64), rev)


def test_sobol_second_dimension_known_points():
    # x -> x + 1 polynomial: 0, 1/2, 3/4, 1/4, 5/8, 1/8, 3/8, 7/8 in index order
    got = oracle.sobol(np.arange(8), 1) / 2.0 ** 32
    np.testing.assert_array_equal(got, [0, 0.5, 0.75, 0.25, 0.625, 0.125, 0.375, 0.875])


@pytest.mark.parametrize("dim", range(9))
def test_sobol_dimensions_are_stratified(dim):
    """The first 2^m points of every dimension put one point in each interval [k/2^m, (k+1)/2^m)."""
    x = oracle.sobol(np.arange(4096), dim).astype(np.uint64)
    for m in range(1, 13):
        cells = x[: 1 << m] >> np.uint64(32 - m)
        assert len(np.unique(cells)) == 1 << m, (dim, m)


def test_sobol_first_two_dimensions_form_a_0m2_net():
    """Every elementary dyadic box of area 2^-10 holds exactly one of the first 1024 points."""
    m = 10
    x0 = oracle.sobol(np.arange(1 << m), 0).astype(np.uint64)
    x1 = oracle.sobol(np.arange(1 << m), 1).astype(np.uint64)
    for a in range(m + 1):
        b = m - a
        cells = (x0 >> np.uint64(32 - a) if a else np.zeros_like(x0)) * np.uint64(1 << b) + \
                (x1 >> np.uint64(32 - b) if b else np.zeros_like(x1))
        assert len(np.unique(cells)) == 1 << m, a


def test_sobol_sampler_uniforms_and_white_furnace():
    u = np.stack([oracle.uniforms(7, s, 99, sampler=1) for s in range(64)])
    assert np.all(u >= 0) and np.all(u < 1) and np.all(np.round(u * 2 ** 24) == u * 2 ** 24)
    # one pixel's 64 samples: per dimension, a rotated stratified set (one point per 1/64 cell after the shift)
    for d in range(9):
        shifted = np.sort((u[:, d] - u[0, d] + oracle.sobol([0], d)[0] / 2.0 ** 32) % 1.0)
        assert len(np.unique(np.floor(shifted * 64 + 1e-9))) == 64
    sc, cam = _furnace_setup()
    out = oracle.render(sc, cam, env_uniform(1.0, 16, 32), spp=16, seed=1,
                        params=dict(brdf_mode=1, sampling_mode=1, sampler=1))
    np.testing.assert_allclose(out["rgb"], 1.0, atol=1e-12)


# ---------------------------------------------------------------- Eq. 6


@pytest.mark.parametrize("o", [0.3, 0.75, 0.99, 0.995, 1.0])
def test_head_on_single_surfel(o):
    """Centre hit: alpha~ = min(0.99, o); rho = alpha a + (1 - alpha) E."""
    a = np.array([0.2, 0.4, 0.6], np.float32).astype(np.float64)  # inputs are FP32
    ch, _ = trace1(make_scene([disk(o=o, a=a)]), (0, 0, 3), (0, 0, -1))
    alpha = min(0.99, float(np.float32(o)))
    assert ch[CH["hits"]] == 1
    assert ch[CH["W"]] == pytest.approx(alpha, abs=1e-14)
    assert ch[CH["T"]] == pytest.approx(1 - alpha, abs=1e-14)
    assert ch[CH["depth"]] == pytest.approx(3.0 * alpha / (alpha + 1e-8), abs=1e-12)
    np.testing.assert_allclose(ch[CH["n0"]:CH["n2"] + 1], [0, 0, 1], atol=1e-15)
    E = float(np.float32(0.7))
    np.testing.assert_allclose(ch[CH["rho0"]:CH["rho2"] + 1], alpha * a + (1 - alpha) * E, atol=1e-12)
    np.testing.assert_allclose(ch[CH["a0"]:CH["a2"] + 1], a * alpha / (alpha + 1e-8), atol=1e-12)


def test_half_opacity_radius():
    """At |xi|^2 = 2 ln 2 the Gaussian response is exactly one half."""
    su = float(np.float32(0.2))
    x0 = su * math.sqrt(2 * math.log(2))
    ch, _ = trace1(make_scene([disk(o=0.8, s=(su, 0.05))]), (x0, 0, 3), (0, 0, -1))
    assert ch[CH["W"]] == pytest.approx(float(np.float32(0.8)) / 2, abs=1e-12)


def test_back_facing_normal_points_at_ray_and_depth_is_ray_distance():
    ch, _ = trace1(make_scene([disk(o=0.9, s=(2.0, 2.0), flip=True)]), (0, 0, 3), (1, 0, -3))
    W = ch[CH["W"]]
    k = W / (W + 1e-8)
    np.testing.assert_allclose(ch[CH["n0"]:CH["n2"] + 1], [0, 0, 1], atol=1e-15)
    assert ch[CH["depth"]] == pytest.approx(math.sqrt(10.0) * k, abs=1e-12)
    np.testing.assert_allclose(ch[CH["x0"]:CH["x2"] + 1], np.array([1.0, 0, 0]) * k, atol=1e-12)


def test_support_edge_and_opacity_threshold():
    s = 0.1
    inside, _ = trace1(make_scene([disk(o=0.9, s=(s, s))]), (2.999 * s, 0, 3), (0, 0, -1))
    outside, mg = trace1(make_scene([disk(o=0.9, s=(s, s))]), (3.001 * s, 0, 3), (0, 0, -1))
    assert inside[CH["hits"]] == 1 and outside[CH["hits"]] == 0
    assert mg[MG["support"]] < 1e-3  # the near-miss is reported as a small margin
    faint, _ = trace1(make_scene([disk(o=0.003)]), (0, 0, 3), (0, 0, -1))
    assert faint[CH["hits"]] == 0  # 0.003 < 1/255
    behind, _ = trace1(make_scene([disk(z=4.0, o=0.9)]), (0, 0, 3), (0, 0, -1))
    assert behind[CH["hits"]] == 0


# ---------------------------------------------------------------- Eq. 7


def test_two_opaque_disks():
    sc = make_scene([disk(z=0.0, o=1.0, s=(1, 1)), disk(z=-1.0, o=1.0, s=(1, 1))])
    ch, _ = trace1(sc, (0, 0, 3), (0, 0, -1))
    assert ch[CH["hits"]] == 2
    assert ch[CH["W"]] == pytest.approx(0.9999, abs=1e-13)
    assert ch[CH["T"]] == pytest.approx(1e-4, abs=1e-13)
    assert ch[CH["depth"]] == pytest.approx((0.99 * 3 + 0.0099 * 4) / (0.9999 + 1e-8), abs=1e-12)


def test_third_disk_at_the_stop_threshold_is_flagged():
    """(1-0.99)^2 sits on T_min: FP64 keeps going, FP32 stops.  The oracle must flag it."""
    sc = make_scene([disk(z=0.0, o=1.0, s=(1, 1)), disk(z=-1.0, o=1.0, s=(1, 1)), disk(z=-2.0, o=1.0, s=(1, 1))])
    ch, mg = trace1(sc, (0, 0, 3), (0, 0, -1))
    assert mg[MG["stop"]] < 1e-9
    assert ch[CH["hits"]] in (2, 3)


def test_early_stop_after_crossing_hit():
    sc = make_scene([disk(z=-0.1 * k, o=1.0, s=(1, 1)) for k in range(6)])
    ch, _ = trace1(sc, (0, 0, 3), (0, 0, -1))
    assert ch[CH["hits"]] == 3  # T = 1e-2, 1e-4(+), 1e-6 < T_min after the third
    assert ch[CH["T"]] == pytest.approx(1e-6, rel=1e-9)


def _independent_trace(scene, o, d, P):
    """Brute force by a different route: 3x3 solve for the plane hit, SVD normal, explicit products."""
    hits = []
    for i in range(scene.n):
        su, sv = scene.scale[i].astype(np.float64)
        tu, tv = scene.tu[i].astype(np.float64), scene.tv[i].astype(np.float64)
        A = np.stack([d, -su * tu, -sv * tv], 1)
        try:
            t, _, _ = np.linalg.solve(A, scene.mu[i].astype(np.float64) - o)
        except np.linalg.LinAlgError:
            continue
        # "projected onto the tangent axes" (the FP32 axes are orthonormal only to
        # ~1e-7, so the solve's own coordinates are not used for u, v)
        q = o + t * d - scene.mu[i].astype(np.float64)
        u, v = q @ tu / su, q @ tv / sv
        r2 = u * u + v * v
        alpha = min(P["alpha_max"], float(scene.opacity[i]) * math.exp(-0.5 * r2))
        if t > P["t_min"] and r2 <= P["support_r2"] and alpha >= P["alpha_min"]:
            nrm = np.linalg.svd(np.stack([tu, tv]))[2][2]
            nrm = nrm if nrm @ d < 0 else -nrm
            hits.append((t, i, alpha, nrm))
    hits.sort(key=lambda h: (h[0], h[1]))
    used, trans = [], []
    for j, h in enumerate(hits):
        T_j = float(np.prod([1 - hh[2] for hh in hits[:j]]))
        used.append(h)
        trans.append(T_j)
        if T_j * (1 - h[2]) < P["T_min"]:
            break
    w = np.array([T * h[2] for T, h in zip(trans, used)])
    Wsum = w.sum()
    T_fin = float(np.prod([1 - h[2] for h in used])) if used else 1.0
    avg = lambda z: (w[:, None] * np.array(z)).sum(0) / (Wsum + P["eps_w"]) if used else np.zeros(np.shape(z)[1:])
    x = [o + h[0] * d for h in used]
    nbar = avg([h[3] for h in used]) if used else -d
    nbar = nbar / np.linalg.norm(nbar) if np.linalg.norm(nbar) > 1e-12 else -d
    a = [scene.albedo[h[1]].astype(np.float64) for h in used]
    return dict(T=T_fin, W=Wsum, depth=float(avg([[h[0]] for h in used])[0]) if used else 0.0,
                x=avg(x) if used else np.zeros(3), n=nbar, a=avg(a) if used else np.zeros(3),
                m=float(avg([[scene.metallic[h[1]]] for h in used])[0]) if used else 0.0,
                r=float(avg([[scene.roughness[h[1]]] for h in used])[0]) if used else 0.0,
                hits=len(used), rho=(w[:, None] * np.array(a)).sum(0) if used else np.zeros(3))


def test_brute_force_tiny_scenes_by_linear_solve():
    P = oracle.default_params()
    rng = np.random.default_rng(7)
    for trial in range(6):
        n = int(rng.integers(2, 9))
        sc = scene_c1(seed=100 + trial).subset(np.arange(n))
        sc.mu = (sc.mu * 0.2).astype(np.float32)
        sc.scale = (sc.scale * 2.0).astype(np.float32)
        o = np.array([0.0, 0.0, 2.0])
        dirs = rng.normal(size=(120, 3)) * [0.05, 0.05, 0.0] + [0, 0, -1]
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        env = env_uniform(0.0, 4, 8)
        ch, mg = oracle.trace_rays(sc, env, np.repeat(o[None], len(dirs), 0), dirs, P)
        n_hit = 0
        for k, d in enumerate(dirs):
            ref = _independent_trace(sc, o, d, P)
            c = ch[k]
            assert c[CH["hits"]] == ref["hits"]
            n_hit += ref["hits"] > 0
            np.testing.assert_allclose(c[CH["T"]], ref["T"], atol=1e-12)
            np.testing.assert_allclose(c[CH["W"]], ref["W"], atol=1e-12)
            np.testing.assert_allclose(c[CH["depth"]], ref["depth"], atol=1e-10)
            np.testing.assert_allclose(c[CH["x0"]:CH["x2"] + 1], ref["x"], atol=1e-10)
            np.testing.assert_allclose(c[CH["n0"]:CH["n2"] + 1], ref["n"], atol=1e-9)
            np.testing.assert_allclose(c[CH["a0"]:CH["a2"] + 1], ref["a"], atol=1e-10)
            np.testing.assert_allclose(c[CH["m"]], ref["m"], atol=1e-10)
            np.testing.assert_allclose(c[CH["r"]], ref["r"], atol=1e-10)
            np.testing.assert_allclose(c[CH["rho0"]:CH["rho2"] + 1], ref["rho"], atol=1e-12)
        assert n_hit > 10


def test_identity_W_equals_one_minus_T_and_bounds():
    sc, cam = scene_c1(), Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 60.0, 64, 64)
    out = oracle.render(sc, cam, env_uniform(1.0, 8, 16), shade=False)
    ch = out["ch"]
    np.testing.assert_allclose(ch[:, CH["W"]] + ch[:, CH["T"]], 1.0, atol=1e-12)
    assert np.all((ch[:, CH["T"]] >= 0) & (ch[:, CH["T"]] <= 1))
    assert np.all((ch[:, CH["hits"]] == 0) == (ch[:, CH["T"]] == 1.0))
    # a stopped ray crossed T_min on its last hit, whose alpha is at most 0.99
    stopped = ch[:, CH["T"]] < 1e-4
    assert np.all(ch[stopped, CH["T"]] >= 1e-6 - 1e-18)


def test_permutation_invariance():
    sc = scene_c1()
    cam = Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 60.0, 24, 24)
    env = env_smooth(1, 16, 32)
    perm = np.random.default_rng(3).permutation(sc.n)
    a = oracle.render(sc, cam, env, spp=2, seed=5)
    b = oracle.render(sc.subset(perm), cam, env, spp=2, seed=5)
    ok = a["margins"][:, MG["tie"]] > 1e-9
    assert ok.mean() > 0.99
    keep = [CH[k] for k in ["T", "W", "depth", "x0", "x1", "x2", "n0", "n1", "n2", "a0", "a1", "a2", "m", "r",
                            "rho0", "rho1", "rho2", "hits"]]
    np.testing.assert_allclose(a["ch"][ok][:, keep], b["ch"][ok][:, keep], atol=1e-12)
    np.testing.assert_allclose(a["rgb"][ok], b["rgb"][ok], atol=1e-10)


# ---------------------------------------------------------------- Eq. 10-11


def _furnace_setup(o=0.7, a=(1.0, 1.0, 1.0), m=0.0, r=0.5):
    sc = make_scene([disk(o=o, s=(0.6, 0.6), a=a, m=m, r=r)])
    cam = Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 20.0, 8, 8)
    return sc, cam


def test_white_furnace_bsdf_sampling_is_exactly_one():
    sc, cam = _furnace_setup()
    out = oracle.render(sc, cam, env_uniform(1.0, 16, 32), spp=16, seed=1,
                        params=dict(brdf_mode=1, sampling_mode=1))
    assert (out["ch"][:, CH["hits"]] > 0).sum() > 40
    np.testing.assert_allclose(out["rgb"], 1.0, atol=1e-12)


@pytest.mark.parametrize("c,a", [(1.0, (1.0, 1.0, 1.0)), (0.6, (0.3, 0.5, 0.8))])
def test_uniform_env_diffuse_mis_expectation(c, a):
    """Uniform E = c, Lambertian albedo a: each pixel's surface term has mean c a."""
    sc, cam = _furnace_setup(a=a)
    out = oracle.render(sc, cam, env_uniform(c, 16, 32), spp=256, seed=2, params=dict(brdf_mode=1))
    ch = out["ch"]
    hit = ch[:, CH["hits"]] > 0
    T = ch[hit, CH["T"]][:, None]
    Y = (out["rgb"][hit] - T * c) / (1 - T)
    mean, sem = Y.mean(0), Y.std(0, ddof=1) / math.sqrt(hit.sum())
    assert np.all(np.abs(mean - c * np.asarray(a)) < 4 * sem + 1e-12)


def _hemisphere_integral(fn, n_th=400, n_ph=800):
    """Midpoint quadrature of fn(w) over the upper (+z) hemisphere."""
    th = (np.arange(n_th) + 0.5) / n_th * (np.pi / 2)
    ph = (np.arange(n_ph) + 0.5) / n_ph * 2 * np.pi
    T, Ph = np.meshgrid(th, ph, indexing="ij")
    w = np.stack([np.sin(T) * np.cos(Ph), np.sin(T) * np.sin(Ph), np.cos(T)], -1).reshape(-1, 3)
    dA = (np.sin(T) * (np.pi / 2 / n_th) * (2 * np.pi / n_ph)).reshape(-1, 1)
    return (fn(w) * dA).sum(0)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_estimator_is_unbiased_against_quadrature(mode):
    """Mean of Eq. 11 over many seeds equals the rendering integral (Eq. 10)."""
    a, m, r, o = np.array([0.8, 0.6, 0.4]), 0.3, 0.45, 0.8
    sc = make_scene([disk(o=o, s=(0.6, 0.6), a=a, m=m, r=r)])
    cam = Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 10.0, 1, 1)  # one pixel, ray straight down
    env = env_smooth(4, 32, 64)
    wo = np.array([0.0, 0.0, 1.0])
    fcosE = lambda w: oracle.brdf(np.array([0, 0, 1.0]), wo, w, a, m, r) * w[:, 2:3] * oracle.env_eval(env, w)[0]
    ref = _hemisphere_integral(fcosE)
    Ed = oracle.env_eval(env, np.array([[0, 0, -1.0]]))[0][0]
    ests = []
    for seed in range(24):
        out = oracle.render(sc, cam, env, spp=1024, seed=seed, params=dict(sampling_mode=mode))
        T = out["ch"][0, CH["T"]]
        ests.append((out["rgb"][0] - T * Ed) / (1 - T))
    ests = np.array(ests)
    mean, sem = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(len(ests))
    assert np.all(np.abs(mean - ref) < 4.5 * sem + 2e-4 * np.abs(ref)), (mean, ref, sem)


# ---------------------------------------------------------------- BRDF


def _rand_dirs(rng, n):
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    w[:, 2] = np.abs(w[:, 2])
    return w


def test_brdf_closed_form_at_unit_roughness():
    """r = 1: D = 1/pi, G1(c) = 2c/(c+1); m = 1 (F0 = a): f = F / (pi (ci+1)(co+1))."""
    rng = np.random.default_rng(0)
    n = np.array([0, 0, 1.0])
    wi, wo = _rand_dirs(rng, 500), _rand_dirs(rng, 500)
    ci, co = wi[:, 2], wo[:, 2]
    f = oracle.brdf(n, wo, wi, np.ones(3), 1.0, 1.0)
    np.testing.assert_allclose(f, (1 / (np.pi * (ci + 1) * (co + 1)))[:, None].repeat(3, 1), rtol=1e-12)
    h = (wi + wo) / np.linalg.norm(wi + wo, axis=1, keepdims=True)
    f0 = oracle.brdf(n, wo, wi, np.zeros(3), 1.0, 1.0)  # F0 = 0: F = (1 - wo.h)^5
    np.testing.assert_allclose(f0[:, 0], (1 - (wo * h).sum(1)) ** 5 / (np.pi * (ci + 1) * (co + 1)), rtol=1e-10,
                               atol=1e-300)


def test_brdf_reciprocity_lambert_mode_and_lower_hemisphere():
    rng = np.random.default_rng(1)
    n = np.array([0, 0, 1.0])
    wi, wo = _rand_dirs(rng, 300), _rand_dirs(rng, 300)
    a = rng.uniform(0, 1, (300, 3))
    m, r = rng.uniform(0, 1, 300), rng.uniform(0.05, 1, 300)
    np.testing.assert_allclose(oracle.brdf(n, wo, wi, a, m, r), oracle.brdf(n, wi, wo, a, m, r), rtol=1e-12)
    np.testing.assert_allclose(oracle.brdf(n, wo, wi, a, m, r, mode=1), a / np.pi, rtol=1e-15)
    below = wi * [1, 1, -1]
    assert np.all(oracle.brdf(n, wo, below, a, m, r) == 0)


@pytest.mark.parametrize("r", [0.05, 0.2, 0.5, 1.0])
def test_ggx_distribution_is_normalised(r):
    """Integral of D(h) (n.h) over the hemisphere of h is 1 (Walter et al. 2007)."""
    f = lambda c: oracle.ggx_D(c, r) * c * 2 * np.pi
    pts = [1 - 10 * r ** 4, 1 - r ** 4] if r < 0.3 else None
    val, _ = integrate.quad(f, 0.0, 1.0, points=pts, limit=400, epsabs=1e-12, epsrel=1e-10)
    assert val == pytest.approx(1.0, abs=2e-7)


@pytest.mark.parametrize("m,r", [(0.0, 0.3), (1.0, 0.2), (1.0, 0.6), (0.5, 1.0), (1.0, 1.0)])
def test_brdf_energy_bound(m, r):
    """The Lambert lobe k_d/pi reflects exactly k_d = a (1 - m); the microfacet
    lobe (F <= 1, Smith G <= 1, normalised D) reflects at most 1.  The
    metallic-roughness model adds the two without a (1 - F) factor, so only
    the lobes are bounded separately."""
    n = np.array([0, 0, 1.0])
    for th in [0.0, 0.7, 1.3]:
        wo = np.array([math.sin(th), 0, math.cos(th)])
        E = _hemisphere_integral(lambda w: oracle.brdf(n, wo, w, np.ones(3), m, r) * w[:, 2:3], 600, 600)
        spec = E - (1.0 - m)
        assert np.all(spec >= -1e-3) and np.all(spec <= 1.0 + 2e-3)
        if m == 1.0 and r == 1.0 and th == 0.0:
            assert spec[0] == pytest.approx(1 - math.log(2), abs=1e-3)


# ---------------------------------------------------------------- samplers


def test_env_tables_are_normalised():
    t = oracle.env_tables(env_smooth(2, 32, 64))
    assert t["cdf_row"][-1] == 1.0 and np.all(t["cdf_col"][:, -1] == 1.0)
    assert np.all(np.diff(t["cdf_row"]) > 0)
    assert t["pmf_row"].sum() == pytest.approx(1.0, abs=1e-14)


def test_env_sampler_matches_its_pmf_and_pdf():
    env = env_smooth(3, 16, 32)
    rng = np.random.default_rng(11)
    u = np.floor(rng.uniform(0, 1, (200_000, 2)) * 2 ** 24) / 2 ** 24
    dirs, pdf = oracle.env_sample(env, u)
    th = np.arccos(np.clip(dirs[:, 1], -1, 1))
    ph = np.arctan2(dirs[:, 0], -dirs[:, 2]) + np.pi
    row = np.clip((th / np.pi * 16).astype(int), 0, 15)
    col = np.clip((ph / (2 * np.pi) * 32).astype(int), 0, 31)
    counts = np.bincount(row * 32 + col, minlength=16 * 32)
    t = oracle.env_tables(env)
    expected = (t["pmf_row"][:, None] * t["pmf_col"]).reshape(-1) * len(u)
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(chi2, 16 * 32 - 1) > 1e-4
    _, pdf_eval = oracle.env_eval(env, dirs)
    np.testing.assert_allclose(pdf, pdf_eval, rtol=1e-6)  # acos round trip near the poles
    # the density integrates to one over the sphere
    w = rng.normal(size=(400_000, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    est = oracle.env_eval(env, w)[1] * 4 * np.pi
    assert abs(est.mean() - 1) < 5 * est.std() / math.sqrt(len(est))


@pytest.mark.parametrize("p_spec,r", [(0.0, 0.5), (0.5, 0.3), (1.0, 0.5)])
def test_bsdf_sampler_density_is_consistent(p_spec, r):
    """E[cos+ / pdf] over the sampler's own draws equals pi (hemisphere integral of cos)."""
    rng = np.random.default_rng(5)
    n = np.array([0.3, -0.2, 0.9])
    n /= np.linalg.norm(n)
    wo = np.array([-0.5, 0.1, 0.8])
    wo /= np.linalg.norm(wo)
    u = np.floor(rng.uniform(0, 1, (400_000, 3)) * 2 ** 24) / 2 ** 24
    wi, pdf = oracle.bsdf_sample(n, wo, r, p_spec, u)
    c = wi @ n
    g = np.where((c > 0) & (pdf > 0), c / np.where(pdf > 0, pdf, 1), 0.0)
    assert abs(g.mean() - np.pi) < 5 * g.std() / math.sqrt(len(g))
    np.testing.assert_allclose(oracle.bsdf_pdf(n, wo, r, p_spec, wi), pdf, rtol=1e-12)
    if p_spec == 0.0:  # Malley: cos^2 of the sampled direction is uniform
        assert stats.kstest(c ** 2, "uniform").pvalue > 1e-4


# ---------------------------------------------------------------- Eq. 2 (rigid object transform)


def _rot_y(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]], np.float32)


def test_rigid_identity_and_untouched_objects():
    sc = scene_c1()
    two = Scene(sc.mu, sc.tu, sc.tv, sc.scale, sc.opacity, sc.albedo, sc.metallic, sc.roughness,
                np.array([0, 400, sc.n], np.int32))
    same = oracle.rigid(two, 1, np.eye(3), np.zeros(3))
    for k in ["mu", "tu", "tv", "scale", "opacity", "albedo", "metallic", "roughness"]:
        np.testing.assert_array_equal(getattr(same, k), getattr(two, k))
    moved = oracle.rigid(two, 1, _rot_y(0.7), np.array([0.3, -0.2, 0.1], np.float32))
    np.testing.assert_array_equal(moved.mu[:400], two.mu[:400])  # object 0 untouched
    assert not np.allclose(moved.mu[400:], two.mu[400:])


def test_rigid_preserves_distances_and_frames():
    sc = scene_c1()
    R, t = _rot_y(1.1), np.array([0.5, 0.25, -0.75], np.float32)
    mv = oracle.rigid(sc, 0, R, t)
    i, j = np.random.default_rng(2).integers(0, sc.n, (2, 200))
    d0 = np.linalg.norm(sc.mu[i].astype(np.float64) - sc.mu[j], axis=1)
    d1 = np.linalg.norm(mv.mu[i].astype(np.float64) - mv.mu[j], axis=1)
    np.testing.assert_allclose(d1, d0, rtol=1e-6, atol=1e-6)
    for a, b in [("tu", "tu"), ("tv", "tv"), ("tu", "tv")]:
        g0 = np.sum(getattr(sc, a).astype(np.float64) * getattr(sc, b), axis=1)
        g1 = np.sum(getattr(mv, a).astype(np.float64) * getattr(mv, b), axis=1)
        np.testing.assert_allclose(g1, g0, atol=1e-6)
    # two moves equal one move by the composed transform (up to one extra FP32 rounding)
    R2, t2 = _rot_y(-0.4), np.array([-0.1, 0.05, 0.2], np.float32)
    twice = oracle.rigid(mv, 0, R2, t2)
    R12 = (R2.astype(np.float64) @ R.astype(np.float64)).astype(np.float32)
    t12 = (R2.astype(np.float64) @ t + t2).astype(np.float32)
    once = oracle.rigid(sc, 0, R12, t12)
    np.testing.assert_allclose(twice.mu, once.mu, atol=3e-6)
    np.testing.assert_allclose(twice.tu, once.tu, atol=3e-6)


def test_moving_scene_and_camera_together_leaves_the_image_unchanged():
    """Under a uniform environment, a rigid move of every object together with
    the camera is a change of frame: the rendered pixels stay the same."""
    sc = scene_c1()
    cam = Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 60.0, 24, 24)
    env = env_uniform(0.8, 8, 16)
    R, t = _rot_y(0.9), np.array([0.4, -0.3, 0.2], np.float32)
    mv = oracle.rigid(sc, 0, R, t)
    R64, t64 = R.astype(np.float64), t.astype(np.float64)
    cam2 = Camera(tuple(R64 @ np.array(cam.eye, float) + t64), tuple(R64 @ np.array(cam.target, float) + t64),
                  tuple(R64 @ np.array(cam.up, float)), cam.fovy_deg, cam.width, cam.height)
    a = oracle.render(sc, cam, env, shade=False)
    b = oracle.render(mv, cam2, env, shade=False)
    ok = (a["margins"].min(axis=1) > 1e-4) & (b["margins"].min(axis=1) > 1e-4)
    assert ok.mean() > 0.8
    for k in ["T", "W", "depth", "a0", "a1", "a2", "rho0", "rho1", "rho2", "hits"]:
        np.testing.assert_allclose(a["ch"][ok, CH[k]], b["ch"][ok, CH[k]], atol=2e-4)


# ---------------------------------------------------------------- Eq. 2 state assembly and its adjoint


def _three_objects():
    sc = scene_c1()
    return Scene(sc.mu, sc.tu, sc.tv, sc.scale, sc.opacity, sc.albedo, sc.metallic, sc.roughness,
                 np.array([0, 300, 650, sc.n], np.int32))


def _flat17(sc):
    return np.concatenate([sc.mu, sc.tu, sc.tv, sc.scale, sc.opacity[:, None], sc.albedo,
                           sc.metallic[:, None], sc.roughness[:, None]], axis=1).astype(np.float64)


_FIELD_OF_COLUMN = [("mu", 0), ("mu", 1), ("mu", 2), ("tu", 0), ("tu", 1), ("tu", 2), ("tv", 0), ("tv", 1),
                    ("tv", 2), ("scale", 0), ("scale", 1), ("opacity", None), ("albedo", 0), ("albedo", 1),
                    ("albedo", 2), ("metallic", None), ("roughness", None)]


def _state_transforms():
    R = np.stack([_rot_y(0.8), _rot_y(-2.3) @ np.array([[1, 0, 0], [0, 0.6, -0.8], [0, 0.8, 0.6]], np.float32)])
    t = np.array([[0.3, -0.1, 0.25], [-0.4, 0.2, 0.05]], np.float32)
    return R.astype(np.float32), t


def test_state_assembly_moves_only_object_centres_and_axes():
    sc = _three_objects()
    R, t = _state_transforms()
    st = oracle.assemble_state(sc, R, t)
    for k in ["scale", "opacity", "albedo", "metallic", "roughness"]:
        np.testing.assert_array_equal(getattr(st, k), getattr(sc, k))
    for k in ["mu", "tu", "tv"]:  # the background B enters every state as it is
        np.testing.assert_array_equal(getattr(st, k)[:300], getattr(sc, k)[:300])
        assert not np.allclose(getattr(st, k)[300:650], getattr(sc, k)[300:650])
    # identity transforms reproduce the canonical scene bit for bit
    same = oracle.assemble_state(sc, np.stack([np.eye(3)] * 2), np.zeros((2, 3)))
    np.testing.assert_array_equal(_flat17(same), _flat17(sc))
    with pytest.raises(ValueError):
        oracle.assemble_state(sc, R[:1], t[:1])


def test_state_pullback_matches_finite_differences_of_the_assembly():
    """The assembly is affine in the canonical parameters, so a central
    difference of <c, S_k(x)> is exact up to the FP32 rounding of the moved
    values; it must reproduce the pulled-back cotangent for every kind of
    entry (moved centres and axes, shared attributes, background)."""
    sc = _three_objects()
    R, t = _state_transforms()
    rng = np.random.default_rng(11)
    c = rng.normal(size=(sc.n, 17))
    g = oracle.state_pullback(sc.object_offsets, R, c)
    h = 2.0 ** -6
    picks = [(i, k) for i in (5, 299, 300, 477, 649, 650, 999) for k in range(17)]
    for i, k in picks:
        field, comp = _FIELD_OF_COLUMN[k]
        vals = []
        for sgn in (1.0, -1.0):
            x = sc.copy()
            arr = getattr(x, field)
            if comp is None:
                arr[i] += np.float32(sgn * h)
            else:
                arr[i, comp] += np.float32(sgn * h)
            vals.append(float(np.sum(c * _flat17(oracle.assemble_state(x, R, t)))))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[i, k]) < 1e-4 * np.abs(c).max(), (i, k, fd, g[i, k])


def test_state_pullback_special_cases():
    sc = _three_objects()
    rng = np.random.default_rng(12)
    c = rng.normal(size=(sc.n, 17))
    # identity transforms: the cotangent passes unchanged
    np.testing.assert_array_equal(oracle.state_pullback(sc.object_offsets, np.stack([np.eye(3)] * 2), c), c)
    # a quarter turn about +y maps canonical +z to world +x and canonical -x to world +z,
    # so world-space gradients along +x and +z pull back to +z and -x
    Q = np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]], np.float32)
    e = np.zeros((sc.n, 17))
    e[400, 0] = 1.0   # d/d mu_x of a surfel of object 1
    e[700, 5] = 1.0   # d/d tu_z of a surfel of object 2
    g = oracle.state_pullback(sc.object_offsets, np.stack([Q, Q]), e)
    np.testing.assert_array_equal(g[400, 0:3], [0.0, 0.0, 1.0])
    np.testing.assert_array_equal(g[700, 3:6], [-1.0, 0.0, 0.0])
    assert np.count_nonzero(g) == 2
