"""Python face of liblightfuse.so: argument marshalling around the C ABI.

Device memory and streams come from PyTorch; every step of the path runs in
the library's CUDA kernels.  There is no CPU fallback: constructing a Tracer
without the built extension or without a CUDA device raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

from . import _native as N

SCENE_FIELDS = ["mu", "tu", "tv", "scale", "opacity", "albedo", "metallic", "roughness"]
SCENE_WIDTH = dict(mu=3, tu=3, tv=3, scale=2, opacity=1, albedo=3, metallic=1, roughness=1)
GRAD_SLICES = dict(mu=(0, 3), tu=(3, 6), tv=(6, 9), scale=(9, 11), opacity=(11, 12), albedo=(12, 15),
                   metallic=(15, 16), roughness=(16, 17))


def default_params(**kw) -> N.LfParams:
    p = N.LfParams()
    _check(N.load().lf_params_default(C.byref(p)))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _check(st, ctx=None):
    if st != N.LF_OK:
        msg = N.load().lf_last_error(ctx).decode() if ctx else ""
        raise N.LightFuseError(st, msg)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def camera_struct(cam) -> N.LfCamera:
    c = N.LfCamera()
    c.eye[:] = [float(v) for v in cam.eye]
    c.target[:] = [float(v) for v in cam.target]
    c.up[:] = [float(v) for v in cam.up]
    c.fovy_deg = float(cam.fovy_deg)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


@dataclass
class SceneTensors:
    """Surfel attributes (Eq. 1) as FP32 CUDA tensors, object k owning
    surfels [object_offsets[k], object_offsets[k+1]) (object 0: background)."""
    mu: torch.Tensor
    tu: torch.Tensor
    tv: torch.Tensor
    scale: torch.Tensor
    opacity: torch.Tensor
    albedo: torch.Tensor
    metallic: torch.Tensor
    roughness: torch.Tensor
    object_offsets: Sequence[int] = field(default_factory=list)

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    @classmethod
    def from_numpy(cls, scene, device="cuda"):
        kw = {k: torch.as_tensor(getattr(scene, k), dtype=torch.float32, device=device).contiguous()
              for k in SCENE_FIELDS}
        return cls(**kw, object_offsets=[int(v) for v in scene.object_offsets])

    def tensors(self):
        return [getattr(self, k) for k in SCENE_FIELDS]


class Tracer:
    """One lf_ctx: a built scene, its BVH and up to 16 environment maps."""

    def __init__(self, params: Optional[N.LfParams] = None, stream: Optional[torch.cuda.Stream] = None, **kw):
        if not torch.cuda.is_available():
            raise RuntimeError("Tracer needs a CUDA device")
        self.lib = N.load()
        self.params = params if params is not None else default_params(**kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(self.lib.lf_create(C.byref(self.params), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.ctx = h
        self.scene: Optional[SceneTensors] = None
        self.envs = {}
        self._counters = None
        self.state_token = 0  # counts lf_state_assemble calls

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        _check(st, self.ctx)

    def sync(self):
        self.check(self.lib.lf_sync(self.ctx))

    # ------------------------------------------------------------ scene
    def build(self, scene: SceneTensors):
        s, arr = self._scene_struct(scene)
        self.check(self.lib.lf_bvh_build(self.ctx, C.byref(s)))
        self.state_token += 1
        self.scene = scene
        self._offsets = list(arr)

    @staticmethod
    def _scene_struct(scene: SceneTensors):
        for k in SCENE_FIELDS:
            t = getattr(scene, k)
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{k}: expected a contiguous float32 CUDA tensor")
            if t.numel() != scene.n * SCENE_WIDTH[k]:
                raise ValueError(f"{k}: expected {scene.n} x {SCENE_WIDTH[k]} values")
        offs = list(scene.object_offsets) or [0, scene.n]
        arr = (C.c_int * len(offs))(*offs)
        return N.LfScene(*[_ptr(getattr(scene, k)) for k in SCENE_FIELDS], scene.n, arr, len(offs) - 1), arr

    def _state_transforms(self, R, t=None):
        m = len(self._offsets) - 2
        Rv = torch.as_tensor(R, dtype=torch.float32).reshape(-1).tolist()
        if len(Rv) != 9 * m:
            raise ValueError(f"expected {m} rotations (objects 1..{m})")
        Rf = (C.c_float * max(1, 9 * m))(*Rv)
        if t is None:
            return Rf, None
        tv = torch.as_tensor(t, dtype=torch.float32).reshape(-1).tolist()
        if len(tv) != 3 * m:
            raise ValueError(f"expected {m} translations (objects 1..{m})")
        return Rf, (C.c_float * max(1, 3 * m))(*tv)

    def assemble_state(self, canonical: SceneTensors, R, t):
        """Eq. 2: write the state whose objects 1..M sit at (R[o-1], t[o-1])
        into the built scene from the canonical (shared) parameters, and refit."""
        s, _keep = self._scene_struct(canonical)
        Rf, tf = self._state_transforms(R, t)
        self.check(self.lib.lf_state_assemble(self.ctx, C.byref(s), Rf, tf))
        self.state_token += 1

    def state_pullback(self, R, d_world: torch.Tensor, d_canonical: torch.Tensor):
        """d_canonical += the state's per-surfel gradient d_world carried back
        through Eq. 2 (both N x 17)."""
        self._check_dev(d_world, d_canonical)
        n = self.scene.n
        if d_world.numel() != n * N.G_STRIDE or d_canonical.numel() != n * N.G_STRIDE:
            raise ValueError(f"expected {n} x {N.G_STRIDE} gradients")
        Rf, _ = self._state_transforms(R)
        self.check(self.lib.lf_state_pullback(self.ctx, Rf, _ptr(d_world), _ptr(d_canonical)))

    def refit(self, object_id: int, R, t):
        Rf = (C.c_float * 9)(*[float(v) for v in torch.as_tensor(R).reshape(-1).tolist()])
        tf = (C.c_float * 3)(*[float(v) for v in torch.as_tensor(t).reshape(-1).tolist()])
        self.check(self.lib.lf_bvh_refit(self.ctx, int(object_id), Rf, tf))
        self.state_token += 1

    def sync_scene(self, object_id: int = -1):
        self.check(self.lib.lf_scene_sync(self.ctx, int(object_id)))

    def set_material(self, object_id: int, rgb=None, metallic: float = -1.0, roughness: float = -1.0):
        c = (C.c_float * 3)(*[float(v) for v in rgb]) if rgb is not None else None
        self.check(self.lib.lf_material_set(self.ctx, int(object_id), c, float(metallic), float(roughness)))

    def set_env(self, env_id: int, rgb: torch.Tensor):
        if rgb.dtype != torch.float32 or rgb.dim() != 3 or rgb.shape[2] != 3:
            raise ValueError("environment: expected an (H, W, 3) float32 CUDA tensor")
        rgb = rgb.contiguous()
        self.check(self.lib.lf_env_set(self.ctx, int(env_id), _ptr(rgb), rgb.shape[0], rgb.shape[1]))
        self.envs[env_id] = rgb

    def env_tables(self, env_id: int):
        e = self.envs[env_id]
        H, W = e.shape[0], e.shape[1]
        out = [torch.empty(H, device=e.device), torch.empty(H, device=e.device),
               torch.empty(H * W, device=e.device), torch.empty(H * W, device=e.device)]
        self.check(self.lib.lf_env_tables(self.ctx, int(env_id), *[_ptr(t) for t in out]))
        return dict(pmf_row=out[0], cdf_row=out[1], pmf_col=out[2].view(H, W), cdf_col=out[3].view(H, W))

    # ------------------------------------------------------------ rendering
    def trace_primary(self, cam, env_id: int = 0, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((N.LF_GBUF_CHANNELS, cam.height, cam.width), device="cuda", dtype=torch.float32)
        c = camera_struct(cam)
        self.check(self.lib.lf_trace_primary(self.ctx, C.byref(c), int(env_id), _ptr(out)))
        return out

    def shade_scratch_bytes(self, cam, spp: int) -> int:
        return int(self.lib.lf_shade_scratch_bytes(cam.width, cam.height, int(spp)))

    def alloc_samples(self, cam, spp: int) -> torch.Tensor:
        """Per-sample buffer of lf_shade_bounce (reusable by backward)."""
        return torch.empty((self.shade_scratch_bytes(cam, spp) + 3) // 4, device="cuda", dtype=torch.float32)

    def shade(self, cam, gbuf: torch.Tensor, env_id: int = 0, spp: int = 16, seed: int = 0,
              out: Optional[torch.Tensor] = None, ray_count: Optional[torch.Tensor] = None,
              samples: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((cam.height, cam.width, 3), device="cuda", dtype=torch.float32)
        if samples is None:
            samples = self.alloc_samples(cam, spp)
        c = camera_struct(cam)
        self.check(self.lib.lf_shade_bounce(self.ctx, C.byref(c), _ptr(gbuf), int(env_id), int(spp),
                                            C.c_uint64(seed), _ptr(out), _ptr(ray_count), _ptr(samples),
                                            samples.numel() * samples.element_size()))
        return out

    def sample_terms(self, cam, gbuf: torch.Tensor, env_id: int, spp: int, samples: torch.Tensor) -> torch.Tensor:
        """(width * height, spp, 3) per-sample terms c_s of the shade() call that filled `samples`."""
        out = torch.empty((cam.width * cam.height, spp, 3), device="cuda", dtype=torch.float32)
        c = camera_struct(cam)
        self.check(self.lib.lf_shade_sample_terms(self.ctx, C.byref(c), _ptr(gbuf), int(env_id), int(spp),
                                                  _ptr(samples), samples.numel() * samples.element_size(),
                                                  _ptr(out)))
        return out

    def scratch_bytes(self, cam, spp: int) -> int:
        return int(self.lib.lf_backward_scratch_bytes(cam.width, cam.height, int(spp)))

    def backward(self, cam, gbuf, env_id, spp, seed, dL_drgb=None, dL_dgbuf=None, d_surfel=None, d_env=None,
                 scratch=None, fwd_samples=None):
        """Accumulates into d_surfel (N, 17) and d_env (H, W, 3); returns them.

        fwd_samples: the `samples` buffer of the matching shade() call (the
        shading adjoint then reuses its frozen data instead of replaying).
        """
        if d_surfel is None:
            d_surfel = torch.zeros((self.scene.n, N.G_STRIDE), device="cuda", dtype=torch.float32)
        if scratch is None and dL_drgb is not None:
            nbytes = (9 * cam.width * cam.height * 4 + 256) if fwd_samples is not None else self.scratch_bytes(cam, spp)
            scratch = torch.empty((nbytes + 3) // 4, device="cuda", dtype=torch.float32)
        c = camera_struct(cam)
        nbytes = scratch.numel() * scratch.element_size() if scratch is not None else 0
        self.check(self.lib.lf_trace_backward(self.ctx, C.byref(c), _ptr(gbuf), int(env_id), int(spp),
                                              C.c_uint64(seed), _ptr(dL_drgb), _ptr(dL_dgbuf), _ptr(d_surfel),
                                              _ptr(d_env), _ptr(fwd_samples), _ptr(scratch), nbytes))
        return d_surfel, d_env

    def set_counters(self, counters: Optional[torch.Tensor]):
        """counters: int64 CUDA tensor of 20 (5 kernel slots x [nodes, tests, composited, rays]) or None."""
        if counters is not None and (not counters.is_cuda or counters.dtype != torch.int64
                                     or not counters.is_contiguous() or counters.numel() < 20):
            raise ValueError("counters must be a contiguous int64 CUDA tensor of at least 20 elements")
        self._counters = counters
        self.check(self.lib.lf_set_counters(self.ctx, _ptr(counters)))

    def profile(self, enable: bool):
        self.check(self.lib.lf_profile(self.ctx, int(bool(enable))))

    def profile_read(self):
        """ms of [primary, gen, NEE shadow, continuation, secondary shadow, combine, shading adjoint,
        adjoint re-traversal] of the last calls (the last two 0 before a profiled backward)."""
        ms = (C.c_float * 8)()
        self.check(self.lib.lf_profile_read(self.ctx, ms))
        return list(ms)

    def geometry_loss(self, cam, gbuf: torch.Tensor, depth_ref: torch.Tensor, depth_conf: torch.Tensor,
                      normal_ref: torch.Tensor, eps: float = 1e-8, weights=(1.0, 1.0, 1.0),
                      dL_dgbuf: Optional[torch.Tensor] = None):
        """Geometry-refinement losses (Eq. 8-9) of one view: returns (L_D, L_N, L_DN) and, when dL_dgbuf (a
        G-buffer-shaped tensor) is given, adds the weighted gradient to its depth and normal planes.
        depth_ref / depth_conf: (H, W); normal_ref: (3, H, W)."""
        for t in (gbuf, depth_ref, depth_conf, normal_ref) + ((dL_dgbuf,) if dL_dgbuf is not None else ()):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("geometry_loss: contiguous float32 CUDA tensors expected")
        c = camera_struct(cam)
        nbytes = int(self.lib.lf_geometry_loss_scratch_bytes(cam.width, cam.height))
        scratch = torch.empty((nbytes + 3) // 4, dtype=torch.float32, device="cuda")
        w = (C.c_float * 3)(*[float(x) for x in weights])
        out = (C.c_double * 3)()
        self.check(self.lib.lf_geometry_loss(self.ctx, C.byref(c), _ptr(gbuf), _ptr(depth_ref), _ptr(depth_conf),
                                             _ptr(normal_ref), C.c_float(eps), w, _ptr(dL_dgbuf), _ptr(scratch),
                                             nbytes, out))  # synchronises: scratch outlives its use
        return tuple(out)

    @staticmethod
    def _check_dev(*ts):
        for t in ts:
            if t is not None and not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("contiguous float32 CUDA tensors expected")

    def opacity_loss(self, cam, gbuf: torch.Tensor, weight: float = 1.0, dL_dgbuf: Optional[torch.Tensor] = None):
        """L_alpha (Eq. 4) on the traced weight sums; adds weight * gradient to dL_dgbuf's W plane."""
        self._check_dev(gbuf, dL_dgbuf)
        c, out = camera_struct(cam), C.c_double()
        self.check(self.lib.lf_opacity_loss(self.ctx, C.byref(c), _ptr(gbuf), C.c_float(weight), _ptr(dL_dgbuf),
                                            C.byref(out)))
        return out.value

    def scale_loss(self, s_max: float, weight: float = 1.0, d_surfel: Optional[torch.Tensor] = None):
        """L_s (Eq. 5) over the scene's scales; adds weight * gradient to d_surfel's scale columns."""
        self._check_dev(self.scene.scale, d_surfel)
        out = C.c_double()
        self.check(self.lib.lf_scale_loss(self.ctx, _ptr(self.scene.scale), int(self.scene.n), C.c_float(s_max),
                                          C.c_float(weight), _ptr(d_surfel), C.byref(out)))
        return out.value

    def env_tv_loss(self, rgb: torch.Tensor, weight: float = 1.0, d_env: Optional[torch.Tensor] = None):
        """L_TV (Eq. 14) of an (H, W, 3) environment map; adds weight * gradient to d_env."""
        self._check_dev(rgb, d_env)
        out = C.c_double()
        self.check(self.lib.lf_env_tv_loss(self.ctx, _ptr(rgb), int(rgb.shape[0]), int(rgb.shape[1]),
                                           C.c_float(weight), _ptr(d_env), C.byref(out)))
        return out.value

    def measure_l2_read(self, nbytes: int = 32 << 20, reps: int = 40) -> float:
        """L2 read bandwidth in GB/s (a measurement helper)."""
        gbs = C.c_float()
        self.check(self.lib.lf_measure_l2_read(self.ctx, C.c_size_t(int(nbytes)), int(reps), C.byref(gbs)))
        return float(gbs.value)

    def philox(self, ctr: torch.Tensor, k0: int, k1: int) -> torch.Tensor:
        out = torch.empty_like(ctr)
        self.check(self.lib.lf_philox(self.ctx, _ptr(ctr), ctr.shape[0], C.c_uint32(k0), C.c_uint32(k1), _ptr(out)))
        return out

    def bvh_wide(self, object_id: int):
        """(slots (cap, WIDE, 8) float32: lo.xyz, code bits, hi.xyz, count bits; root code, root count):
        the object's wide BVH storage."""
        import numpy as np
        cap, root, rcount, wide = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self.check(self.lib.lf_bvh_copy_wide(self.ctx, int(object_id), None, 0, C.byref(cap), C.byref(root),
                                             C.byref(rcount), C.byref(wide)))
        buf = np.zeros((max(1, cap.value), 2, wide.value, 4), np.float32)  # per node: lo quads, hi quads
        self.check(self.lib.lf_bvh_copy_wide(self.ctx, int(object_id), buf.ctypes.data_as(C.c_void_p), buf.nbytes,
                                             C.byref(cap), C.byref(root), C.byref(rcount), C.byref(wide)))
        slots = np.ascontiguousarray(buf.transpose(0, 2, 1, 3)).reshape(-1, wide.value, 8)
        return slots[: cap.value], root.value, rcount.value

    def bvh_nodes(self, object_id: int):
        n_int, root = C.c_int(), C.c_int()
        self.check(self.lib.lf_bvh_info(self.ctx, int(object_id), C.byref(n_int), C.byref(root)))
        import numpy as np
        buf = np.zeros((max(1, n_int.value), 16), np.float32)
        self.check(self.lib.lf_bvh_copy_nodes(self.ctx, int(object_id), buf.ctypes.data_as(C.c_void_p),
                                              buf.nbytes))
        return buf[: n_int.value], root.value


def split_surfel_grad(d_surfel: torch.Tensor):
    """(N, 17) gradient -> dict of per-attribute gradients."""
    return {k: d_surfel[:, a:b].reshape(-1) if b - a == 1 else d_surfel[:, a:b] for k, (a, b) in GRAD_SLICES.items()}
