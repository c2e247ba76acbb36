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
# Per shading sample: a shading ray starts from the record's position with
# its residual (x + x_lo, within ~3e-10 of the FP64 composite at the median
# pixel and ~1e-7 at the 99th percentile, where a pixel blends surfaces a
# distance apart and the FP32 opacities of the weights count) along a
# direction assembled in double-float from the record's normal and roughness with
# their residuals and rounded once to FP32 (measured against the oracle on
# C2 and C4: 2e-8 rad at the median, 6e-8 at the 99th percentile).  Its
# support, opacity and depth-order decisions are flagged when a ray shift of
# SHIFT (the oracle's *_shift margins, a direction change counted as
# (1 + t) times an origin shift) flips them; on those runs no unflagged
# sample differed by more than 1e-4 with half this SHIFT either.  Also the
# relative margins of the primary ray for the FP32 storage of the records; a
# uniform within FP32 rounding (2^-24) of an environment CDF entry (FP32
# tables may select the neighbouring texel), a continuation direction within
# 1e-6 rad of a texel edge of the piecewise-constant environment pdf.
SHIFT = 1e-7
FLAG_SAMPLE = dict(support=1e-6, alpha=1e-6, tmin=1e-3, tie=1e-9, stop=2e-5, cos=2e-6, frame=2e-6, cdf=6e-8,
                   ptex=1e-6, support_shift=SHIFT, alpha_shift=SHIFT, tie_shift=SHIFT)


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


def sample_flags(o, kinds=FLAG, kinds_sample=FLAG_SAMPLE):
    """(n, spp) bool: shading sample s of pixel i is flagged when the pixel's
    primary ray is flagged or one of the sample's own decisions (or the
    pixel-level shading decisions folded into every sample) is."""
    fp = flagged(o["margins"], kinds)
    ms = o["margins_sample"]
    f = np.zeros(ms.shape[:2], bool)
    for k, thr in kinds_sample.items():
        f |= ms[:, :, MG[k]] < thr
    return f | fp[:, None]


def compare_samples(o, terms_gpu, T_gpu, rgb_gpu, spp, tol=1e-4, kinds_sample=FLAG_SAMPLE):
    """Per-sample comparison of the shading estimator (Eq. 11).

    Each sample's share of its pixel, (1 - T) / spp * c_s, is compared with
    the oracle's on every unflagged sample:
        |d| <= tol * max(1, |share|)       (unclamped, HDR)
    and each pixel with the flagged samples removed on both sides,
        L' = L - (1 - T) / spp * sum_{s flagged} c_s,
    on every pixel whose primary ray is not flagged:
        |dL'| <= tol * max(1, |L'|)  and  |clip(L', 0, 1) - ...| <= tol.
    terms_gpu: (n, spp, 3) GPU terms c_s; T_gpu: (n,) GPU transmittance;
    rgb_gpu: (n, 3) GPU pixel values.  Returns a dict of the measured
    fractions and worst errors (asserts nothing)."""
    fs = sample_flags(o, kinds_sample=kinds_sample)
    fp = flagged(o["margins"])
    k = (1.0 - o["ch"][:, OCH["T"]]) / spp
    kg = (1.0 - np.asarray(T_gpu, np.float64)) / spp
    so = k[:, None, None] * o["samples"]
    sg = kg[:, None, None] * np.asarray(terms_gpu, np.float64)
    rel = np.abs(sg - so) / np.maximum(1.0, np.abs(so))
    ok = ~fs
    Lo = o["rgb"] - (so * fs[:, :, None]).sum(1)
    Lg = np.asarray(rgb_gpu, np.float64) - (sg * fs[:, :, None]).sum(1)
    pok = ~fp
    prel = (np.abs(Lg - Lo) / np.maximum(1.0, np.abs(Lo)))[pok]
    pcl = np.abs(np.clip(Lg, 0, 1) - np.clip(Lo, 0, 1))[pok]
    return dict(flagged_samples=float(fs.mean()), n_samples=int(fs.size), flagged_pixels=float(fp.mean()),
                n_pixels=int(len(fp)),
                sample_rel=float(rel[ok].max()) if ok.any() else 0.0,
                failing_samples=int(((rel > tol) & ok[:, :, None]).any(2).sum()),
                pixel_rel=float(prel.max()) if prel.size else 0.0,
                pixel_clamped=float(pcl.max()) if pcl.size else 0.0)


def gpu_shaded(tr, cam, env_id, spp, seed, pix):
    """Trace and shade one frame on the GPU; returns (G-buffer tensor, sample
    buffer, G-buffer (n, C), per-sample terms (n, spp, 3), rgb (n, 3)) with
    the last three at the flat pixel indices `pix`."""
    import torch
    g = tr.trace_primary(cam, env_id)
    samples = tr.alloc_samples(cam, spp)
    rgb = tr.shade(cam, g, env_id, spp=spp, seed=seed, samples=samples)
    terms = tr.sample_terms(cam, g, env_id, spp, samples)
    tr.sync()
    pt = torch.as_tensor(np.asarray(pix, np.int64), device="cuda")
    return g, samples, gbuf_at(g, pix), terms[pt].cpu().numpy(), rgb.reshape(-1, 3)[pt].cpu().numpy()


def assert_shading(r, tol=1e-4, max_flagged=0.01):
    """The per-sample comparison's bounds: flagged fractions under
    `max_flagged` (at least one sample or pixel may be flagged in a tiny
    image), no unflagged sample or pixel beyond `tol`."""
    assert r["flagged_pixels"] * r["n_pixels"] <= max(1.0, max_flagged * r["n_pixels"]), r
    assert r["flagged_samples"] * r["n_samples"] <= max(1.0, max_flagged * r["n_samples"]), r
    assert r["failing_samples"] == 0 and r["sample_rel"] <= tol, r
    assert r["pixel_rel"] <= tol and r["pixel_clamped"] <= tol, r
