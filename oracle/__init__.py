"""FP64 CPU oracle for the surfel ray tracer (TEST INFRASTRUCTURE ONLY).

The slow, plain brute-force reference the CUDA path is checked against: every
ray against every surfel, a full sort of the accepted hits, Eq. 6-7
compositing, the one-bounce estimator of Eq. 11 and a reverse-mode FP64
gradient under the path-replay freeze of Sec. 3.3.  Only `tests/`, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product
path never does.  It shares no code with the CUDA library.

Readings of points the paper leaves open are the defaults of `default_params`
(support radius 3 sigma, opacity threshold 1/255, eps = 1e-8, early stop at
T < 1e-4 after the crossing hit, t_min = 1e-4, ray offset 1e-3 along the
composited normal, specular-lobe probability 0.5).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lf_oracle.cpp")
_LIB = os.path.join(_HERE, "liblf_oracle.so")

# Per-pixel channel layout of the oracle's outputs.
CHANNELS = ["T", "W", "depth", "x0", "x1", "x2", "n0", "n1", "n2", "a0", "a1", "a2", "m", "r",
            "rho0", "rho1", "rho2", "nlen", "hits", "t_stop", "id_stop", "sig"]
NDIFF = 17  # channels 0..16 are differentiable
MARGINS = ["support", "alpha", "cap", "tmin", "tie", "stop", "cos", "frame", "cdf", "ptex", "support_shift",
           "alpha_shift", "tie_shift"]
PARAM_ORDER = ["mu", "tu", "tv", "scale", "opacity", "albedo", "metallic", "roughness"]


def default_params(**kw):
    p = dict(T_min=1e-4, alpha_min=1.0 / 255.0, alpha_max=0.99, support_r2=9.0, eps_w=1e-8,
             t_min=1e-4, ray_offset=1e-3, p_spec=0.5, brdf_mode=0, sampling_mode=0, sampler=0)
    p.update(kw)
    return p


def build(force: bool = False) -> str:
    """Compile lf_oracle.cpp into liblf_oracle.so (g++, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared",
                               "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_float)) for k in PARAM_ORDER] + [("n", C.c_int)]


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("target", C.c_double * 3), ("up", C.c_double * 3),
                ("fovy_deg", C.c_double), ("width", C.c_int), ("height", C.c_int)]


class _Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in ["T_min", "alpha_min", "alpha_max", "support_r2", "eps_w",
                                          "t_min", "ray_offset", "p_spec"]] + \
               [("brdf_mode", C.c_int), ("sampling_mode", C.c_int), ("sampler", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (test use: a test plants a
    mistake in the text and checks that a pin catches it)."""
    src = out_path + ".cpp"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", src,
                           "-o", out_path])
    return out_path


class using:
    """Context manager: route this module's calls to another build of the
    oracle (a `compile_variant` output) and back."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = _declare(C.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _declare(L):
    """Argument and result types of the C interface on a loaded library."""
    dp, fp, ip, u32p = (C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int), C.POINTER(C.c_uint32))
    L.or_render.restype = C.c_int64
    L.or_render.argtypes = [C.POINTER(_Scene), C.POINTER(_Scene), C.POINTER(_Camera), fp, fp, C.c_int,
                            C.c_int, C.POINTER(_Params), ip, C.c_int, C.c_int, C.c_uint64, C.c_int, dp,
                            dp, dp, C.c_int, dp, dp]
    L.or_grad.restype = None
    L.or_grad.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), fp, C.c_int, C.c_int,
                          C.POINTER(_Params), ip, C.c_int, C.c_int, C.c_uint64, C.c_int, dp, dp, dp, dp,
                          C.c_int]
    L.or_trace_rays.argtypes = [C.POINTER(_Scene), fp, C.c_int, C.c_int, C.POINTER(_Params), dp, dp,
                                C.c_int, dp, dp]
    L.or_shadow_rays.argtypes = [C.POINTER(_Scene), C.POINTER(_Params), dp, dp, C.c_int, dp]
    L.or_philox.argtypes = [u32p, C.c_int, C.c_uint32, C.c_uint32, u32p]
    L.or_uniforms.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_int, dp]
    L.or_sobol.argtypes = [u32p, C.c_int, C.c_int, u32p]
    L.or_env_tables.argtypes = [fp, C.c_int, C.c_int, dp, dp, dp, dp]
    L.or_env_sample.argtypes = [fp, C.c_int, C.c_int, dp, C.c_int, dp, dp]
    L.or_env_eval.argtypes = [fp, C.c_int, C.c_int, dp, C.c_int, dp, dp]
    L.or_brdf.argtypes = [dp, dp, dp, dp, dp, dp, C.c_int, C.c_int, dp]
    L.or_bsdf_sample.argtypes = [dp, dp, C.c_double, C.c_double, dp, C.c_int, dp, dp]
    L.or_ggx_D.restype = C.c_double
    L.or_ggx_D.argtypes = [C.c_double, C.c_double]
    L.or_bsdf_pdf.argtypes = [dp, dp, C.c_double, C.c_double, dp, C.c_int, dp]
    L.or_camera_dirs.argtypes = [C.POINTER(_Camera), C.POINTER(C.c_int), C.c_int, dp]
    return L


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _SceneHandle:
    """Keeps the float32 arrays alive while the C struct points at them."""

    def __init__(self, scene):
        self.arrays = [_f32(getattr(scene, k)) for k in PARAM_ORDER]
        self.s = _Scene(*[_p(a, C.c_float) for a in self.arrays], scene.n)


def _camera(cam):
    # the camera reaches the renderer as FP32 values
    f = lambda v: [float(np.float32(x)) for x in v]
    return _Camera((C.c_double * 3)(*f(cam.eye)), (C.c_double * 3)(*f(cam.target)), (C.c_double * 3)(*f(cam.up)),
                   float(np.float32(cam.fovy_deg)), int(cam.width), int(cam.height))


def _params(p):
    p = default_params(**(p or {}))
    return _Params(*[float(p[k]) for k in ["T_min", "alpha_min", "alpha_max", "support_r2", "eps_w", "t_min",
                                           "ray_offset", "p_spec"]], int(p["brdf_mode"]), int(p["sampling_mode"]),
                   int(p["sampler"]))


def render(scene, cam, env, pixels=None, spp=0, seed=0, shade=True, params=None, scene0=None, env0=None,
           threads=0):
    """Render camera pixels.

    Returns dict(ch=(n,NCH), rgb=(n,3), margins=(n,NM) of the primary ray,
    margins_shade=(n,NM) of all shading rays of each pixel, rays=int) and,
    when shading, the per-sample terms of Eq. 11: samples=(n,spp,3) (c_s, so
    that rgb = T E(d) + (1 - T)/spp * sum_s c_s) and margins_sample=(n,spp,NM)
    (each sample's own decisions plus the pixel-level shading decisions).

    scene0/env0: parameters the frozen path-replay data come from (default:
    the same as scene/env).
    """
    L = lib()
    if pixels is None:
        pixels = np.arange(cam.width * cam.height, dtype=np.int32)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    n = len(pixels)
    sh = _SceneHandle(scene)
    sh0 = _SceneHandle(scene0) if scene0 is not None else sh
    rgb_env = _f32(env.rgb)
    rgb_env0 = _f32(env0.rgb) if env0 is not None else rgb_env
    ch = np.zeros((n, len(CHANNELS)), np.float64)
    rgb = np.zeros((n, 3), np.float64)
    mg = np.zeros((n, 2, len(MARGINS)), np.float64)
    per = bool(shade) and spp > 0
    srgb = np.zeros((n, spp, 3), np.float64) if per else None
    smg = np.zeros((n, spp, len(MARGINS)), np.float64) if per else None
    cam_c = _camera(cam)
    prm = _params(params)
    rays = L.or_render(C.byref(sh.s), C.byref(sh0.s), C.byref(cam_c), _p(rgb_env, C.c_float),
                       _p(rgb_env0, C.c_float), env.height, env.width, C.byref(prm), _p(pixels, C.c_int), n,
                       int(spp), C.c_uint64(seed), int(bool(shade)), _p(ch, C.c_double), _p(rgb, C.c_double),
                       _p(mg, C.c_double), int(threads), _p(srgb, C.c_double) if per else None,
                       _p(smg, C.c_double) if per else None)
    out = dict(ch=ch, rgb=rgb, margins=mg[:, 0].copy(), margins_shade=mg[:, 1].copy(), rays=int(rays))
    if per:
        out.update(samples=srgb, margins_sample=smg)
    return out


def grad(scene, cam, env, pixels, spp, seed, dL_drgb=None, dL_dch=None, shade=True, params=None, threads=0):
    """Gradient of sum(dL_drgb*rgb) + sum(dL_dch*ch[:, :17]) (path-replay freeze).

    Returns (d_surfel (N,17) in the order mu3 tu3 tv3 s2 o a3 m r, d_env (H,W,3)).
    """
    L = lib()
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    n = len(pixels)
    sh = _SceneHandle(scene)
    rgb_env = _f32(env.rgb)
    d_s = np.zeros((scene.n, 17), np.float64)
    d_e = np.zeros((env.height, env.width, 3), np.float64)
    g_rgb = _f64(dL_drgb) if dL_drgb is not None else None
    g_ch = _f64(dL_dch) if dL_dch is not None else None
    if g_rgb is not None:
        assert g_rgb.shape == (n, 3)
    if g_ch is not None:
        assert g_ch.shape == (n, NDIFF)
    cam_c = _camera(cam)
    prm = _params(params)
    L.or_grad(C.byref(sh.s), C.byref(cam_c), _p(rgb_env, C.c_float), env.height, env.width, C.byref(prm),
              _p(pixels, C.c_int), n, int(spp), C.c_uint64(seed), int(bool(shade)),
              _p(g_rgb, C.c_double) if g_rgb is not None else None,
              _p(g_ch, C.c_double) if g_ch is not None else None,
              _p(d_s, C.c_double), _p(d_e, C.c_double), int(threads))
    return d_s, d_e


def camera_dirs(cam, pixels=None):
    """(n, 3) ray directions of camera pixels (FP64 pinhole direction rounded once to FP32)."""
    L = lib()
    if pixels is None:
        pixels = np.arange(cam.width * cam.height, dtype=np.int32)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    out = np.zeros((len(pixels), 3), np.float64)
    cam_c = _camera(cam)
    L.or_camera_dirs(C.byref(cam_c), _p(pixels, C.c_int), len(pixels), _p(out, C.c_double))
    return out


def rigid(scene, k, R, t):
    """Eq. 2 on object k: a copy of `scene` with mu <- R mu + t, tu <- R tu,
    tv <- R tv for the object's surfels (scales, opacity and materials are
    unchanged).  The scene stores FP32 values, so each component is evaluated
    in FP64 as ((R0 x0 + R1 x1) + R2 x2) (+ t) -- every product of two FP32
    values is exact -- and rounded once to FP32."""
    out = scene.copy()
    lo, hi = int(scene.object_offsets[k]), int(scene.object_offsets[k + 1])
    R = np.asarray(R, np.float32).astype(np.float64).reshape(3, 3)
    t = np.asarray(t, np.float32).astype(np.float64).reshape(3)
    for name, shift in (("mu", True), ("tu", False), ("tv", False)):
        x = getattr(scene, name)[lo:hi].astype(np.float64)
        y = np.empty_like(x)
        for r in range(3):
            acc = (R[r, 0] * x[:, 0] + R[r, 1] * x[:, 1]) + R[r, 2] * x[:, 2]
            y[:, r] = acc + t[r] if shift else acc
        getattr(out, name)[lo:hi] = y.astype(np.float32)
    return out


def assemble_state(canonical, R, t):
    """Eq. 2: the scene S_k of one state from the shared canonical scene.  The
    background (object 0) enters as it is; object o = 1..M is placed by
    T_{k,o} = (R[o-1], t[o-1]) acting on its centres and tangent axes only,
    evaluated as `rigid` does (FP64, one rounding per component)."""
    R = np.asarray(R, np.float32).reshape(-1, 3, 3)
    t = np.asarray(t, np.float32).reshape(-1, 3)
    M = canonical.n_objects - 1
    if len(R) != M or len(t) != M:
        raise ValueError(f"need {M} object transforms")
    out = canonical.copy()
    for o in range(1, M + 1):
        out = rigid(out, o, R[o - 1], t[o - 1])
    return out


def state_pullback(object_offsets, R, d_world):
    """Adjoint of `assemble_state` (chain rule through Eq. 2): the gradient of
    the canonical parameters given the gradient d_world (n, 17) of the state's
    parameters, in the per-surfel layout mu 3 | tu 3 | tv 3 | scale 2 |
    opacity | albedo 3 | metallic | roughness.  For a surfel of object o >= 1
    the mu, tu and tv triples g become R^T g, (R^T g)_j = (R_0j g_0 + R_1j g_1)
    + R_2j g_2 in FP64 (t drops out: it does not depend on the surfel); every
    other entry, and every entry of the background, passes unchanged."""
    R = np.asarray(R, np.float32).astype(np.float64).reshape(-1, 3, 3)
    g = np.asarray(d_world, np.float64).reshape(-1, 17)
    out = g.copy()
    off = np.asarray(object_offsets)
    if len(R) != len(off) - 2:
        raise ValueError(f"need {len(off) - 2} object transforms")
    for o in range(1, len(off) - 1):
        lo, hi = int(off[o]), int(off[o + 1])
        Ro = R[o - 1]
        for a in (0, 3, 6):
            x = g[lo:hi, a:a + 3]
            for j in range(3):
                out[lo:hi, a + j] = (Ro[0, j] * x[:, 0] + Ro[1, j] * x[:, 1]) + Ro[2, j] * x[:, 2]
    return out


def trace_rays(scene, env, origins, dirs, params=None):
    """Eq. 6-7 composite of explicit rays.  Returns (ch (n,NCH), margins (n,8))."""
    L = lib()
    o, d = _f64(origins).reshape(-1, 3), _f64(dirs).reshape(-1, 3)
    n = len(o)
    sh = _SceneHandle(scene)
    rgb_env = _f32(env.rgb)
    ch = np.zeros((n, len(CHANNELS)))
    mg = np.zeros((n, len(MARGINS)))
    prm = _params(params)
    L.or_trace_rays(C.byref(sh.s), _p(rgb_env, C.c_float), env.height, env.width, C.byref(prm),
                    _p(o, C.c_double), _p(d, C.c_double), n, _p(ch, C.c_double), _p(mg, C.c_double))
    return ch, mg


def shadow_rays(scene, origins, dirs, params=None):
    L = lib()
    o, d = _f64(origins).reshape(-1, 3), _f64(dirs).reshape(-1, 3)
    v = np.zeros(len(o))
    sh = _SceneHandle(scene)
    prm = _params(params)
    L.or_shadow_rays(C.byref(sh.s), C.byref(prm), _p(o, C.c_double), _p(d, C.c_double), len(o),
                     _p(v, C.c_double))
    return v


def philox(counters, key0, key1):
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    lib().or_philox(_p(c, C.c_uint32), len(c), C.c_uint32(key0), C.c_uint32(key1), _p(out, C.c_uint32))
    return out


def uniforms(pixel, sample, seed, sampler=0):
    u = np.zeros(9)
    lib().or_uniforms(C.c_uint32(pixel), C.c_uint32(sample), C.c_uint64(seed), int(sampler), _p(u, C.c_double))
    return u


def sobol(index, dim):
    """32-bit Sobol fractions of dimension `dim` (0-8) for integer indices."""
    idx = np.ascontiguousarray(index, dtype=np.uint32)
    out = np.zeros(len(idx), np.uint32)
    lib().or_sobol(_p(idx, C.c_uint32), len(idx), int(dim), _p(out, C.c_uint32))
    return out


def env_tables(env):
    H, W = env.height, env.width
    rgb = _f32(env.rgb)
    out = [np.zeros(H), np.zeros(H), np.zeros((H, W)), np.zeros((H, W))]
    lib().or_env_tables(_p(rgb, C.c_float), H, W, *[_p(a, C.c_double) for a in out])
    return dict(pmf_row=out[0], cdf_row=out[1], pmf_col=out[2], cdf_col=out[3])


def env_sample(env, u):
    u = _f64(u).reshape(-1, 2)
    rgb = _f32(env.rgb)
    dirs = np.zeros((len(u), 3))
    pdf = np.zeros(len(u))
    lib().or_env_sample(_p(rgb, C.c_float), env.height, env.width, _p(u, C.c_double), len(u),
                        _p(dirs, C.c_double), _p(pdf, C.c_double))
    return dirs, pdf


def env_eval(env, dirs):
    d = _f64(dirs).reshape(-1, 3)
    rgb = _f32(env.rgb)
    val = np.zeros((len(d), 3))
    pdf = np.zeros(len(d))
    lib().or_env_eval(_p(rgb, C.c_float), env.height, env.width, _p(d, C.c_double), len(d),
                      _p(val, C.c_double), _p(pdf, C.c_double))
    return val, pdf


def brdf(n, wo, wi, a, m, r, mode=0):
    n, wo, wi, a = (_f64(x).reshape(-1, 3) for x in (n, wo, wi, a))
    cnt = max(len(n), len(wo), len(wi), len(a))
    n, wo, wi, a = (np.ascontiguousarray(np.broadcast_to(x, (cnt, 3))) for x in (n, wo, wi, a))
    m = np.ascontiguousarray(np.broadcast_to(_f64(m).reshape(-1), (cnt,)))
    r = np.ascontiguousarray(np.broadcast_to(_f64(r).reshape(-1), (cnt,)))
    out = np.zeros((cnt, 3))
    lib().or_brdf(*[_p(x, C.c_double) for x in (n, wo, wi, a, m, r)], cnt, int(mode), _p(out, C.c_double))
    return out


def ggx_D(nh, r):
    return lib().or_ggx_D(float(nh), float(r))


def bsdf_sample(n, wo, r, p_spec, u):
    u = _f64(u).reshape(-1, 3)
    n, wo = _f64(n).reshape(3), _f64(wo).reshape(3)
    wi = np.zeros((len(u), 3))
    pdf = np.zeros(len(u))
    lib().or_bsdf_sample(_p(n, C.c_double), _p(wo, C.c_double), float(r), float(p_spec), _p(u, C.c_double),
                         len(u), _p(wi, C.c_double), _p(pdf, C.c_double))
    return wi, pdf


def bsdf_pdf(n, wo, r, p_spec, wi):
    wi = _f64(wi).reshape(-1, 3)
    n, wo = _f64(n).reshape(3), _f64(wo).reshape(3)
    pdf = np.zeros(len(wi))
    lib().or_bsdf_pdf(_p(n, C.c_double), _p(wo, C.c_double), float(r), float(p_spec), _p(wi, C.c_double),
                      len(wi), _p(pdf, C.c_double))
    return pdf
