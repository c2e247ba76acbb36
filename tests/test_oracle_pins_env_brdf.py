"""Pins of the oracle's environment lookup (Eq. 10-11: E(w) read from an
equirectangular map) and of its microfacet terms (Sec. 3.3 BRDF, citing
Walter et al. 2007), each against a fact other than the oracle's own formula:

  * environment lookup: the value at each texel centre is that texel; halfway
    between two texel centres it is their mean; the azimuth wraps at
    phi = 0 / 2 pi and the polar angle clamps at the poles; the axis
    directions land on the texels the mapping convention (row 0 looks up
    along +y, phi = 0 at +z, phi increasing towards -x) predicts;
  * Smith G1 against the Lambda form G1 = 1 / (1 + Lambda),
    Lambda = (-1 + sqrt(1 + alpha_g^2 tan^2 theta)) / 2, at r < 1 where the
    (1 - alpha_g^2) term of the oracle's form does not vanish;
  * the Schlick F0 blend F0 = 0.04 (1 - m) + a m and the GGX peak
    D(n.h = 1) = 1 / (pi alpha_g^2) in a closed-form mirror configuration.

Each pin is also run against a copy of the oracle with the matching
plausible mistake planted (a dropped half-texel offset, a wrapped instead of
clamped pole, alpha_g in place of alpha_g^2 inside G1), and must fail there.
"""
import math
import os

import numpy as np
import pytest

import oracle
from synthetic.scenes import EnvMap

H, W = 16, 32


def _dir(theta, phi):
    """Unit direction with polar angle theta from +y and azimuth phi, phi = 0
    at +z and phi = pi / 2 at -x (the map's column order)."""
    st = np.sin(theta)
    return np.stack([-st * np.sin(phi), np.cos(theta) * np.ones_like(phi), st * np.cos(phi)], -1)


def _ramp():
    r, c = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    rgb = np.stack([1.0 + r * W + c, 1.0 + r, 1.0 + c], -1).astype(np.float32)
    return EnvMap(rgb)


def _lookup(env, dirs):
    return oracle.env_eval(env, np.asarray(dirs, np.float64).reshape(-1, 3))[0]


def check_texel_centres():
    env = _ramp()
    r, c = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    th = np.pi * (r.ravel() + 0.5) / H
    ph = 2 * np.pi * (c.ravel() + 0.5) / W
    got = _lookup(env, _dir(th, ph))
    np.testing.assert_allclose(got, env.rgb.reshape(-1, 3), rtol=1e-9, atol=0)


def check_midpoints_give_means():
    env = _ramp()
    rgb = env.rgb.astype(np.float64)
    # halfway in azimuth between (r, c) and (r, c + 1), inside the map
    r, c = np.meshgrid(np.arange(H), np.arange(W - 1), indexing="ij")
    got = _lookup(env, _dir(np.pi * (r.ravel() + 0.5) / H, 2 * np.pi * (c.ravel() + 1.0) / W))
    np.testing.assert_allclose(got, 0.5 * (rgb[r, c] + rgb[r, c + 1]).reshape(-1, 3), rtol=1e-9)
    # halfway in polar angle between (r, c) and (r + 1, c)
    r, c = np.meshgrid(np.arange(H - 1), np.arange(W), indexing="ij")
    got = _lookup(env, _dir(np.pi * (r.ravel() + 1.0) / H, 2 * np.pi * (c.ravel() + 0.5) / W))
    np.testing.assert_allclose(got, 0.5 * (rgb[r, c] + rgb[r + 1, c]).reshape(-1, 3), rtol=1e-9)


def check_azimuth_wraps():
    env = _ramp()
    rgb = env.rgb.astype(np.float64)
    rows = np.arange(H)
    th = np.pi * (rows + 0.5) / H
    # phi = 0 (the +z half-plane) sits between the last and the first column
    got = _lookup(env, _dir(th, np.zeros(H)))
    np.testing.assert_allclose(got, 0.5 * (rgb[rows, W - 1] + rgb[rows, 0]), rtol=1e-9)
    # a quarter texel on either side of phi = 0
    q = 0.25 * 2 * np.pi / W
    np.testing.assert_allclose(_lookup(env, _dir(th, np.full(H, q))), 0.25 * rgb[rows, W - 1] + 0.75 * rgb[rows, 0],
                               rtol=1e-9)
    np.testing.assert_allclose(_lookup(env, _dir(th, np.full(H, -q))), 0.75 * rgb[rows, W - 1] + 0.25 * rgb[rows, 0],
                               rtol=1e-9)


def check_poles_clamp():
    env = _ramp()
    rgb = env.rgb.astype(np.float64)
    cols = np.arange(W)
    ph = 2 * np.pi * (cols + 0.5) / W
    eps = 0.25 * np.pi / H  # a quarter texel from the pole: beyond the first row centre
    np.testing.assert_allclose(_lookup(env, _dir(np.full(W, eps), ph)), rgb[0, cols], rtol=1e-9)
    np.testing.assert_allclose(_lookup(env, _dir(np.full(W, np.pi - eps), ph)), rgb[H - 1, cols], rtol=1e-9)


def check_axis_directions():
    """The mapping convention as texels: a map lit in one texel is seen from
    the axis direction the convention names and from no other axis."""
    axes = {"+y": (0, 1, 0), "-y": (0, -1, 0), "+z": (0, 0, 1), "-z": (0, 0, -1), "+x": (1, 0, 0), "-x": (-1, 0, 0)}
    cases = [  # lit texel -> axis that sees it with bilinear weight 1/4 (equator: between rows H/2-1, H/2)
        ((H // 2, 3 * W // 4), "+x", 0.25),
        ((H // 2, W // 4), "-x", 0.25),
        ((H // 2, W // 2), "-z", 0.25),
        ((H // 2, 0), "+z", 0.25),
    ]
    for (r, c), seen, w in cases:
        rgb = np.zeros((H, W, 3), np.float32)
        rgb[r, c] = 1.0
        vals = {k: _lookup(EnvMap(rgb), [v])[0, 0] for k, v in axes.items()}
        assert vals[seen] == pytest.approx(w, abs=1e-12), (r, c, vals)
        assert all(abs(v) < 1e-12 for k, v in vals.items() if k != seen), (r, c, vals)
    # the first row is seen looking up (+y), the last looking down (-y)
    for r, seen in ((0, "+y"), (H - 1, "-y")):
        rgb = np.zeros((H, W, 3), np.float32)
        rgb[r, :] = 1.0
        assert _lookup(EnvMap(rgb), [axes[seen]])[0, 0] == pytest.approx(1.0, abs=1e-12)
        other = "-y" if seen == "+y" else "+y"
        assert abs(_lookup(EnvMap(rgb), [axes[other]])[0, 0]) < 1e-12


ENV_CHECKS = [check_texel_centres, check_midpoints_give_means, check_azimuth_wraps, check_poles_clamp,
              check_axis_directions]


@pytest.mark.parametrize("check", ENV_CHECKS, ids=lambda f: f.__name__)
def test_env_lookup(check):
    check()


# ---------------------------------------------------------------- BRDF


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _g1_lambda(c, alpha_g):
    """Smith G1 from the Lambda form (Walter et al. 2007; Heitz 2014)."""
    tan2 = (1.0 - c * c) / (c * c)
    lam = (-1.0 + np.sqrt(1.0 + alpha_g ** 2 * tan2)) / 2.0
    return 1.0 / (1.0 + lam)


def check_smith_g1_below_unit_roughness():
    """m = 1 and a = 1 make F = 1 and the Lambert lobe 0, so
    f = D G1(wi) G1(wo) / (4 ci co); dividing by the separately pinned D
    (or_ggx_D, normalised by quadrature) leaves the Smith product."""
    rng = np.random.default_rng(3)
    n = np.array([0.0, 0.0, 1.0])
    for r in (0.05, 0.3, 0.7):
        th_i, th_o = rng.uniform(0.05, 1.45, 40), rng.uniform(0.05, 1.45, 40)
        ph = rng.uniform(0, 2 * np.pi, 40)
        wi = np.stack([np.sin(th_i) * np.cos(ph), np.sin(th_i) * np.sin(ph), np.cos(th_i)], 1)
        wo = np.stack([np.sin(th_o), np.zeros(40), np.cos(th_o)], 1)
        f = oracle.brdf(n, wo, wi, np.ones(3), 1.0, r)[:, 0]
        h = _unit(wi + wo)
        D = np.array([oracle.ggx_D(x, r) for x in h[:, 2]])
        G = f * 4 * wi[:, 2] * wo[:, 2] / D
        expect = _g1_lambda(wi[:, 2], r * r) * _g1_lambda(wo[:, 2], r * r)
        np.testing.assert_allclose(G, expect, rtol=1e-10)


def check_f0_blend_and_ggx_peak():
    """Mirror configuration wi = wo = n: n.h = o.h = 1, so F = F0, G1 = 1 and
    f = a (1 - m) / pi + F0 D(1) / 4 with D(1) = 1 / (pi r^4)."""
    n = np.array([0.0, 0.0, 1.0])
    a = np.array([0.2, 0.4, 0.6])
    for r in (0.3, 0.5, 0.9):
        f0 = oracle.brdf(n, n, n, a, 0.0, r)[0]
        np.testing.assert_allclose(f0, a / np.pi + 0.04 / (4 * np.pi * r ** 4), rtol=1e-12)
        f1 = oracle.brdf(n, n, n, a, 1.0, r)[0]
        np.testing.assert_allclose(f1, a / (4 * np.pi * r ** 4), rtol=1e-12)
        fh = oracle.brdf(n, n, n, a, 0.5, r)[0]
        np.testing.assert_allclose(fh, 0.5 * a / np.pi + (0.02 + 0.5 * a) / (4 * np.pi * r ** 4), rtol=1e-12)


BRDF_CHECKS = [check_smith_g1_below_unit_roughness, check_f0_blend_and_ggx_peak]


@pytest.mark.parametrize("check", BRDF_CHECKS, ids=lambda f: f.__name__)
def test_brdf(check):
    check()


# ---------------------------------------------------------------- planted mistakes

SRC = os.path.join(os.path.dirname(oracle.__file__), "lf_oracle.cpp")
MUTANTS = {
    # u without the half-texel offset (texel corners taken as centres)
    "half_texel_u": ([("e.W - 0.5, v =", "e.W, v =")], [check_texel_centres, check_midpoints_give_means,
                                                        check_azimuth_wraps]),
    # v without the half-texel offset
    "half_texel_v": ([("th / PI * e.H - 0.5;", "th / PI * e.H;")], [check_texel_centres, check_poles_clamp]),
    # the polar angle wrapped like the azimuth instead of clamped
    "wrapped_pole": ([("long y0c = std::min<long>(e.H - 1, std::max<long>(0, y0)), "
                       "y1c = std::min<long>(e.H - 1, std::max<long>(0, y0 + 1));",
                       "long y0c = ((y0 % e.H) + e.H) % e.H, y1c = (((y0 + 1) % e.H) + e.H) % e.H;")],
                     [check_poles_clamp]),
    # azimuth measured the other way round
    "mirrored_phi": ([("ph = std::atan2(w.x, -w.z) + PI;", "ph = std::atan2(-w.x, -w.z) + PI;")],
                     [check_axis_directions]),
    # alpha_g in place of alpha_g^2 inside Smith G1
    "g1_alpha": ([("sqrt(a2 + (1.0 - a2) * ci * ci)", "sqrt(ag + (1.0 - ag) * ci * ci)"),
                  ("sqrt(a2 + (1.0 - a2) * co * co)", "sqrt(ag + (1.0 - ag) * co * co)")],
                 [check_smith_g1_below_unit_roughness]),
    # F0 of a dielectric taken as 0.05
    "f0": ([("0.04 * one_m + a.x * m, 0.04 * one_m + a.y * m, 0.04 * one_m + a.z * m",
             "0.05 * one_m + a.x * m, 0.05 * one_m + a.y * m, 0.05 * one_m + a.z * m")],
           [check_f0_blend_and_ggx_peak]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(name, tmp_path):
    edits, checks = MUTANTS[name]
    text = open(SRC).read()
    for old, new in edits:
        assert text.count(old) == 1, old
        text = text.replace(old, new)
    lib = oracle.compile_variant(text, str(tmp_path / f"liblf_oracle_{name}.so"))
    with oracle.using(lib):
        for check in checks:
            with pytest.raises(AssertionError):
                check()
    # and the unmodified oracle passes the same checks
    for check in checks:
        check()
