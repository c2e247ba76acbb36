"""Shared helpers of the GPU tests: build the extension, run both sides on
the same seeded inputs, and flag pixels whose result sits on a discontinuity.

Flags come from the oracle's per-pixel margins (distance of every decision
that could change the result to its threshold): FP32 and FP64 may
legitimately take different branches there, so those pixels are counted and
reported, not compared.
"""
import numpy as np

import oracle

MG = {n: i for i, n in enumerate(oracle.MARGINS)}
OCH = {n: i for i, n in enumerate(oracle.CHANNELS)}

# Relative margins under which a pixel is flagged.
#  Primary rays are the same FP32 ray on both sides and the kernel evaluates
#  depth and u^2 + v^2 in double-float, so only FP32 storage of the packed
#  axes (~1e-7), the FP32 exp and the FP32 transmittance product remain.
#  Shading rays start from an FP32 composite and FP32-sampled directions
#  (~1e-7 relative), which moves hit points by up to ~3e-5 of the smallest
#  surfel scale.
FLAG = dict(support=1e-6, alpha=1e-6, tmin=1e-5, tie=1e-9, stop=2e-5, cos=2e-6, frame=2e-6)
FLAG_SHADE = dict(support=4e-5, alpha=4e-5, tmin=1e-3, tie=1e-8, stop=2e-5, cos=2e-6, frame=2e-6)


def flagged(margins, kinds=FLAG, margins_shade=None, kinds_shade=FLAG_SHADE):
    f = np.zeros(len(margins), bool)
    for k, thr in kinds.items():
        f |= margins[:, MG[k]] < thr
    if margins_shade is not None:
        for k, thr in kinds_shade.items():
            f |= margins_shade[:, MG[k]] < thr
    return f


# G-buffer channel pairs (gpu plane, oracle column)
GBUF_PAIRS = [("T", 0, "T"), ("W", 1, "W"), ("depth", 2, "depth"),
              ("x0", 3, "x0"), ("x1", 4, "x1"), ("x2", 5, "x2"),
              ("n0", 6, "n0"), ("n1", 7, "n1"), ("n2", 8, "n2"),
              ("a0", 9, "a0"), ("a1", 10, "a1"), ("a2", 11, "a2"),
              ("m", 12, "m"), ("r", 13, "r"), ("rho0", 14, "rho0"), ("rho1", 15, "rho1"), ("rho2", 16, "rho2")]


def gpu_tracer(scene, envs, **params):
    import torch
    from paper_2608_29269_b300 import SceneTensors, Tracer
    from paper_2608_29269_b300.build import build
    build()
    tr = Tracer(**params)
    st = SceneTensors.from_numpy(scene)
    tr.build(st)
    for i, e in enumerate(envs):
        tr.set_env(i, torch.as_tensor(e.rgb, device="cuda"))
    return tr, st


def gbuf_at(gbuf, pixels):
    """(C, H, W) tensor -> (len(pixels), C) numpy at flat pixel indices."""
    g = gbuf.reshape(gbuf.shape[0], -1).cpu().numpy()
    return g[:, pixels].T.astype(np.float64)


def compare_gbuf(g_gpu, o_ch, ok, tol=1e-4):
    """Max abs error per channel over the unflagged pixels; returns dict."""
    out = {}
    for name, gi, oname in GBUF_PAIRS:
        d = np.abs(g_gpu[ok, gi] - o_ch[ok, OCH[oname]])
        out[name] = float(d.max()) if d.size else 0.0
    return out
