"""torch.autograd.Function around lf_trace_primary / lf_shade_bounce /
lf_trace_backward (the hand-written adjoint; no autograd tape is recorded
for the renderer itself)."""
from __future__ import annotations

import torch

from . import _native as N
from .tracer import GRAD_SLICES, SCENE_FIELDS, Tracer


class SurfelRender(torch.autograd.Function):
    """rgb, gbuf = SurfelRender.apply(tracer, cam, env_id, spp, seed, env_rgb, *scene_tensors)

    The scene tensors must be the ones the tracer was built with (the kernels
    read the packed BVH records of those tensors).  Gradients flow to every
    surfel attribute and to the environment texels under the path-replay
    freeze of the shading (Sec. 3.3).
    """

    @staticmethod
    def forward(ctx, tracer: Tracer, cam, env_id: int, spp: int, seed: int, env_rgb, *scene):
        gbuf = tracer.trace_primary(cam, env_id)
        samples = tracer.alloc_samples(cam, spp)
        rgb = tracer.shade(cam, gbuf, env_id, spp, seed, samples=samples)
        ctx.tracer, ctx.cam, ctx.env_id, ctx.spp, ctx.seed = tracer, cam, env_id, spp, seed
        ctx.save_for_backward(gbuf, env_rgb, samples)
        ctx.mark_non_differentiable(gbuf)
        return rgb, gbuf

    @staticmethod
    def backward(ctx, g_rgb, g_gbuf):
        gbuf, env_rgb, samples = ctx.saved_tensors
        tr = ctx.tracer
        d_surfel = torch.zeros((tr.scene.n, N.G_STRIDE), device=gbuf.device, dtype=torch.float32)
        d_env = torch.zeros_like(env_rgb) if ctx.needs_input_grad[5] else None
        tr.backward(ctx.cam, gbuf, ctx.env_id, ctx.spp, ctx.seed,
                    dL_drgb=g_rgb.contiguous() if g_rgb is not None else None,
                    dL_dgbuf=None, d_surfel=d_surfel, d_env=d_env, fwd_samples=samples)
        grads = []
        for k in SCENE_FIELDS:
            a, b = GRAD_SLICES[k]
            t = getattr(tr.scene, k)
            grads.append(d_surfel[:, a:b].reshape(t.shape))
        return (None, None, None, None, None, d_env, *grads)


class StateRender(torch.autograd.Function):
    """rgb, gbuf = StateRender.apply(tracer, canonical, R, t, cam, env_id, spp, seed, env_rgb, *canonical.tensors())

    Cross-state supervision (Sec. 3.2): state k of the shared canonical scene
    is assembled by Eq. 2 (objects 1..M at (R[o-1], t[o-1])) into the scene
    the tracer was built on, rendered, and its gradient carried back to the
    canonical parameters, so the residuals of every state accumulate on the
    same surfels.  The backward re-assembles its state when another state was
    assembled since its forward.
    """

    @staticmethod
    def forward(ctx, tracer: Tracer, canonical, R, t, cam, env_id: int, spp: int, seed: int, env_rgb, *params):
        tracer.assemble_state(canonical, R, t)
        token = tracer.state_token
        gbuf = tracer.trace_primary(cam, env_id)
        samples = tracer.alloc_samples(cam, spp)
        rgb = tracer.shade(cam, gbuf, env_id, spp, seed, samples=samples)
        ctx.tracer, ctx.canonical, ctx.R, ctx.t, ctx.token = tracer, canonical, R, t, token
        ctx.cam, ctx.env_id, ctx.spp, ctx.seed = cam, env_id, spp, seed
        ctx.save_for_backward(gbuf, env_rgb, samples)
        ctx.mark_non_differentiable(gbuf)
        return rgb, gbuf

    @staticmethod
    def backward(ctx, g_rgb, g_gbuf):
        gbuf, env_rgb, samples = ctx.saved_tensors
        tr = ctx.tracer
        if tr.state_token != ctx.token:
            tr.assemble_state(ctx.canonical, ctx.R, ctx.t)
        d_world = torch.zeros((tr.scene.n, N.G_STRIDE), device=gbuf.device, dtype=torch.float32)
        d_env = torch.zeros_like(env_rgb) if ctx.needs_input_grad[8] else None
        tr.backward(ctx.cam, gbuf, ctx.env_id, ctx.spp, ctx.seed,
                    dL_drgb=g_rgb.contiguous() if g_rgb is not None else None,
                    dL_dgbuf=None, d_surfel=d_world, d_env=d_env, fwd_samples=samples)
        d_can = torch.zeros_like(d_world)
        tr.state_pullback(ctx.R, d_world, d_can)
        grads = []
        for k in SCENE_FIELDS:
            a, b = GRAD_SLICES[k]
            grads.append(d_can[:, a:b].reshape(getattr(ctx.canonical, k).shape))
        return (None, None, None, None, None, None, None, None, d_env, *grads)


def render_state(tracer: Tracer, canonical, R, t, cam, env_id: int = 0, spp: int = 16, seed: int = 0):
    return StateRender.apply(tracer, canonical, R, t, cam, env_id, spp, seed, tracer.envs[env_id],
                             *canonical.tensors())


def render(tracer: Tracer, cam, env_id: int = 0, spp: int = 16, seed: int = 0):
    s = tracer.scene
    return SurfelRender.apply(tracer, cam, env_id, spp, seed, tracer.envs[env_id], *s.tensors())


def spp_schedule(iteration: int) -> int:
    """Samples per pixel of the inverse-rendering schedule (Sec. 4.2): 8, then
    16 from iteration 7,500 and 32 from iteration 12,000."""
    if iteration < 0:
        raise ValueError("iteration must be non-negative")
    return 8 if iteration < 7500 else (16 if iteration < 12000 else 32)


def trainable_groups(iteration: int):
    """Parameter groups the inverse-rendering stages optimise (Sec. 4.2):
    lighting only until iteration 2,000, lighting and base colour until 9,000,
    then lighting and every material parameter."""
    if iteration < 0:
        raise ValueError("iteration must be non-negative")
    if iteration < 2000:
        return ("env",)
    if iteration < 9000:
        return ("env", "albedo")
    return ("env", "albedo", "metallic", "roughness")
