"""Seeded synthetic scenes, environment maps and cameras.

The paper's datasets (Blender rooms with movable objects, captured rooms) are
not available, so every workload is synthetic and shaped like them: a room
shell (the shared background B of Eq. 2) plus movable objects O_o, each made of
oriented 2D Gaussian surfels (Eq. 1), lit by equirectangular HDR environment
maps.

Conventions of the arrays (all float32, C-contiguous):
  mu (N,3)       surfel centres
  tu, tv (N,3)   tangent axes (unit, orthogonal; tu x tv is the surfel normal)
  scale (N,2)    in-plane scales (s_u, s_v) > 0
  opacity (N,)   o in [0,1]
  albedo (N,3)   base colour a in [0,1]^3
  metallic (N,)  m in [0,1]
  roughness (N,) r in [0,1]
  object_offsets (n_objects+1,) int: object k owns surfels
                 [offsets[k], offsets[k+1]); object 0 is the background.
Environment maps are (H, W, 3) float32, row 0 looking up (+y).

Nothing in this module traces, shades or differentiates; it only draws inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass
class Scene:
    mu: np.ndarray
    tu: np.ndarray
    tv: np.ndarray
    scale: np.ndarray
    opacity: np.ndarray
    albedo: np.ndarray
    metallic: np.ndarray
    roughness: np.ndarray
    object_offsets: np.ndarray = field(default_factory=lambda: np.zeros(2, np.int32))

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    @property
    def n_objects(self) -> int:
        return int(len(self.object_offsets) - 1)

    def arrays(self):
        return dict(mu=self.mu, tu=self.tu, tv=self.tv, scale=self.scale,
                    opacity=self.opacity, albedo=self.albedo,
                    metallic=self.metallic, roughness=self.roughness)

    def copy(self) -> "Scene":
        return Scene(**{k: v.copy() for k, v in self.arrays().items()},
                     object_offsets=self.object_offsets.copy())

    def subset(self, idx, keep_objects: bool = False) -> "Scene":
        """Surfels idx as one object, or (keep_objects, idx sorted) each in its
        original object."""
        idx = np.asarray(idx)
        if keep_objects:
            if np.any(np.diff(idx) <= 0):
                raise ValueError("keep_objects needs sorted, distinct indices")
            offs = np.searchsorted(idx, self.object_offsets).astype(np.int32)
        else:
            offs = np.array([0, len(idx)], np.int32)
        return Scene(**{k: np.ascontiguousarray(v[idx]) for k, v in self.arrays().items()}, object_offsets=offs)


@dataclass
class Camera:
    eye: tuple
    target: tuple
    up: tuple
    fovy_deg: float
    width: int
    height: int

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclass
class EnvMap:
    rgb: np.ndarray  # (H, W, 3) float32

    @property
    def height(self) -> int:
        return int(self.rgb.shape[0])

    @property
    def width(self) -> int:
        return int(self.rgb.shape[1])


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def quat_to_axes(q: np.ndarray):
    """Unit quaternions (w,x,y,z) -> first two columns of the rotation matrix."""
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    c0 = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], 1)
    c1 = np.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], 1)
    return c0, c1


def _frame_from_normal(n: np.ndarray, rng: np.random.Generator):
    """Tangent pair (tu, tv) with tu x tv = n and a random in-plane angle."""
    ref = np.where(np.abs(n[:, 1:2]) < 0.9, np.array([[0.0, 1.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]))
    t1 = np.cross(ref, n)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(n, t1)
    ang = rng.uniform(0.0, 2 * np.pi, size=(n.shape[0], 1))
    tu = np.cos(ang) * t1 + np.sin(ang) * t2
    tv = -np.sin(ang) * t1 + np.cos(ang) * t2
    return tu, tv


def random_surfels(n: int, seed: int = 0) -> Scene:
    """Config 'plain forward': n random surfels in the unit cube.

    centres U[-0.5,0.5]^3, random unit-quaternion axes, scales log-uniform in
    [0.01,0.1], opacity U[0.2,1], albedo U[0,1]^3, metallic U[0,1], roughness
    U[0.05,1].
    """
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-0.5, 0.5, size=(n, 3))
    q = rng.normal(size=(n, 4))
    tu, tv = quat_to_axes(q)
    scale = np.exp(rng.uniform(np.log(0.01), np.log(0.1), size=(n, 2)))
    opacity = rng.uniform(0.2, 1.0, size=n)
    albedo = rng.uniform(0.0, 1.0, size=(n, 3))
    metallic = rng.uniform(0.0, 1.0, size=n)
    roughness = rng.uniform(0.05, 1.0, size=n)
    return Scene(_f32(mu), _f32(tu), _f32(tv), _f32(scale), _f32(opacity), _f32(albedo),
                 _f32(metallic), _f32(roughness), np.array([0, n], np.int32))


def _materials(n, base_albedo, base_metal, base_rough, rng):
    a = np.clip(np.asarray(base_albedo)[None, :] + rng.uniform(-0.05, 0.05, size=(n, 3)), 0.0, 1.0)
    m = np.clip(base_metal + rng.uniform(-0.05, 0.05, size=n), 0.0, 1.0)
    r = np.clip(base_rough + rng.uniform(-0.05, 0.05, size=n), 0.05, 1.0)
    return a, m, r


_FACE_COLOURS = [(0.55, 0.45, 0.35), (0.75, 0.72, 0.68), (0.70, 0.75, 0.80),
                 (0.80, 0.70, 0.60), (0.65, 0.70, 0.65), (0.72, 0.68, 0.75)]


def box_shell(per_face: int, half: float = 2.0, seed: int = 0,
              scale_range=(0.02, 0.04)):
    """Room shell [-half,half]^3: per_face surfels on each face, normals inward."""
    rng = np.random.default_rng(seed)
    parts = []
    for face in range(6):
        axis, sgn = face // 2, (-1.0 if face % 2 == 0 else 1.0)
        pts = rng.uniform(-half, half, size=(per_face, 3))
        pts[:, axis] = sgn * half
        inward = np.zeros((per_face, 3))
        inward[:, axis] = -sgn
        tu, tv = _frame_from_normal(inward, rng)
        sc = np.exp(rng.uniform(np.log(scale_range[0]), np.log(scale_range[1]), size=(per_face, 2)))
        op = rng.uniform(0.6, 1.0, size=per_face)
        base_metal = 0.0 if face != 2 else 0.2  # floor (y = -half) slightly glossy
        a, m, r = _materials(per_face, _FACE_COLOURS[face], base_metal, 0.7 if face != 2 else 0.35, rng)
        parts.append((pts, tu, tv, sc, op, a, m, r))
    return parts


def _shape_points(kind: str, count: int, size: float, rng: np.random.Generator):
    """Area-uniform points and outward normals on a primitive centred at 0."""
    if kind == "sphere":
        r = 0.4 * size
        n = rng.normal(size=(count, 3))
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        return n * r, n, 4 * np.pi * r * r, r
    if kind == "torus":
        R, r = 0.4 * size, 0.15 * size
        out_p, out_n, got = [], [], 0
        while got < count:
            m = 2 * (count - got) + 64
            th = rng.uniform(0, 2 * np.pi, m)
            ph = rng.uniform(0, 2 * np.pi, m)
            keep = rng.uniform(0, 1, m) < (R + r * np.cos(ph)) / (R + r)
            th, ph = th[keep], ph[keep]
            p = np.stack([(R + r * np.cos(ph)) * np.cos(th), r * np.sin(ph),
                          (R + r * np.cos(ph)) * np.sin(th)], 1)
            nn = np.stack([np.cos(ph) * np.cos(th), np.sin(ph), np.cos(ph) * np.sin(th)], 1)
            out_p.append(p)
            out_n.append(nn)
            got += len(p)
        return (np.concatenate(out_p)[:count], np.concatenate(out_n)[:count],
                4 * np.pi * np.pi * R * r, r)
    if kind == "box":
        h = 0.35 * size
        face = rng.integers(0, 6, size=count)
        p = rng.uniform(-h, h, size=(count, 3))
        nn = np.zeros((count, 3))
        ax, sg = face // 2, np.where(face % 2 == 0, -1.0, 1.0)
        p[np.arange(count), ax] = sg * h
        nn[np.arange(count), ax] = sg
        return p, nn, 24 * h * h, h
    if kind == "cylinder":
        r, hh = 0.3 * size, 0.4 * size
        side, cap = 2 * np.pi * r * 2 * hh, np.pi * r * r
        part = rng.uniform(0, side + 2 * cap, size=count)
        th = rng.uniform(0, 2 * np.pi, size=count)
        p = np.zeros((count, 3))
        nn = np.zeros((count, 3))
        s_m = part < side
        p[s_m] = np.stack([r * np.cos(th[s_m]), rng.uniform(-hh, hh, s_m.sum()), r * np.sin(th[s_m])], 1)
        nn[s_m] = np.stack([np.cos(th[s_m]), np.zeros(s_m.sum()), np.sin(th[s_m])], 1)
        c_m = ~s_m
        rad = r * np.sqrt(rng.uniform(0, 1, c_m.sum()))
        top = np.where(part[c_m] < side + cap, 1.0, -1.0)
        p[c_m] = np.stack([rad * np.cos(th[c_m]), top * hh, rad * np.sin(th[c_m])], 1)
        nn[c_m] = np.stack([np.zeros(c_m.sum()), top, np.zeros(c_m.sum())], 1)
        return p, nn, side + 2 * cap, hh
    raise ValueError(kind)


_OBJECT_MATERIALS = {
    "sphere": ((0.85, 0.2, 0.15), 0.0, 0.3),
    "torus": ((0.9, 0.75, 0.3), 0.9, 0.25),
    "box": ((0.2, 0.45, 0.8), 0.1, 0.6),
    "cylinder": ((0.3, 0.75, 0.35), 0.5, 0.45),
}


def object_surfels(kind: str, count: int, centre_xz, floor_y: float, size: float, seed: int):
    """One movable object: `count` surfels on a primitive resting on the floor."""
    rng = np.random.default_rng(seed)
    p, nn, area, extent_y = _shape_points(kind, count, size, rng)
    centre = np.array([centre_xz[0], floor_y + extent_y, centre_xz[1]])
    tu, tv = _frame_from_normal(nn, rng)
    s0 = np.sqrt(area / count)
    sc = s0 * np.exp(rng.uniform(np.log(0.9), np.log(1.1), size=(count, 2)))
    op = rng.uniform(0.6, 1.0, size=count)
    base = _OBJECT_MATERIALS[kind]
    a, m, r = _materials(count, *base, rng)
    return (p + centre, tu, tv, sc, op, a, m, r)


def _assemble(parts_per_object) -> Scene:
    cols = [[], [], [], [], [], [], [], []]
    offsets = [0]
    for obj_parts in parts_per_object:
        n_obj = 0
        for part in obj_parts:
            for i in range(8):
                cols[i].append(part[i])
            n_obj += len(part[0])
        offsets.append(offsets[-1] + n_obj)
    arr = [np.concatenate(c) for c in cols]
    return Scene(_f32(arr[0]), _f32(arr[1]), _f32(arr[2]), _f32(arr[3]), _f32(arr[4]),
                 _f32(arr[5]), _f32(arr[6]), _f32(arr[7]), np.array(offsets, np.int32))


def scene_c1(seed: int = 0) -> Scene:
    """1,000 random surfels in the unit cube (plain forward workload)."""
    return random_surfels(1000, seed)


def scene_c2(seed: int = 0, per_face: int = 10_000, per_object: int = 35_000) -> Scene:
    """Room shell (6 x per_face) plus sphere/torus/box/cylinder (per_object each)."""
    shell = box_shell(per_face, 2.0, seed)
    kinds = ["sphere", "torus", "box", "cylinder"]
    centres = [(-0.8, -0.8), (0.8, -0.8), (-0.8, 0.8), (0.8, 0.8)]
    objs = [[object_surfels(k, per_object, c, -2.0, 1.0, seed * 1000 + 17 * (i + 1))]
            for i, (k, c) in enumerate(zip(kinds, centres))]
    return _assemble([shell] + objs)


def scene_c4(seed: int = 0, n_total: int = 1_000_000, per_face: int = 40_000, n_obj: int = 12) -> Scene:
    """Room shell (6 x per_face) plus n_obj objects sharing the remaining surfels."""
    shell = box_shell(per_face, 2.0, seed)
    rest = n_total - 6 * per_face
    counts = [rest // n_obj] * n_obj
    counts[-1] += rest - sum(counts)
    kinds = ["sphere", "torus", "box", "cylinder"]
    xs, zs = [-1.35, -0.45, 0.45, 1.35], [-1.2, 0.0, 1.2]
    objs = []
    for i in range(n_obj):
        c = (xs[i % 4], zs[(i // 4) % 3])
        objs.append([object_surfels(kinds[i % 4], counts[i], c, -2.0, 0.7, seed * 1000 + 31 * (i + 1))])
    return _assemble([shell] + objs)


def camera_c1(width: int = 64, height: int = 64) -> Camera:
    return Camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height)


def camera_c2(width: int = 800, height: int = 800) -> Camera:
    return Camera((0.0, -0.5, 1.8), (0.0, -1.5, 0.0), (0.0, 1.0, 0.0), 60.0, width, height)


def camera_c4(width: int = 1024, height: int = 1024) -> Camera:
    return Camera((0.0, -0.2, 1.9), (0.0, -1.5, -0.2), (0.0, 1.0, 0.0), 60.0, width, height)


def scene_c3_subset(scene: Scene, cam: Camera, n: int = 512, seed: int = 0, keep_objects: bool = False) -> Scene:
    """First n surfels of a seeded permutation whose centres lie in the view
    cone (as one object, or each in its original object)."""
    rng = np.random.default_rng(seed)
    eye = np.asarray(cam.eye)
    fwd = np.asarray(cam.target) - eye
    fwd /= np.linalg.norm(fwd)
    v = scene.mu.astype(np.float64) - eye
    cosang = (v @ fwd) / np.linalg.norm(v, axis=1)
    inside = np.nonzero(cosang > np.cos(np.radians(0.45 * cam.fovy_deg)))[0]
    pick = rng.permutation(inside)[:n]
    return scene.subset(np.sort(pick), keep_objects=keep_objects)


def perturb_scene(scene: Scene, seed: int = 1, sigma_mu: float = 0.01, shift: float = 0.1) -> Scene:
    """Differentiation target: position noise, roughness and albedo shifted."""
    rng = np.random.default_rng(seed)
    s = scene.copy()
    s.mu = _f32(s.mu + rng.normal(0.0, sigma_mu, size=s.mu.shape))
    s.roughness = _f32(np.clip(s.roughness + shift, 0.05, 1.0))
    s.albedo = _f32(np.clip(s.albedo + shift, 0.0, 1.0))
    return s


def rigid_motion(rng: np.random.Generator, pivot, max_shift: float = 0.5):
    """Rotation about +y through `pivot` and an x/z shift U[-max_shift, max_shift].

    Returns (R, t) for the world-space map x -> R x + t.
    """
    ang = rng.uniform(0.0, 2 * np.pi)
    c, s = np.cos(ang), np.sin(ang)
    R = np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])
    shift = np.array([rng.uniform(-max_shift, max_shift), 0.0, rng.uniform(-max_shift, max_shift)])
    pivot = np.asarray(pivot, np.float64)
    t = pivot + shift - R @ pivot
    return R.astype(np.float32), t.astype(np.float32)


def pixel_subset(width: int, height: int, count: int, seed: int = 0) -> np.ndarray:
    """Sorted, distinct, seeded pixel indices p = y*width + x."""
    rng = np.random.default_rng(seed)
    count = min(count, width * height)
    return np.sort(rng.choice(width * height, size=count, replace=False)).astype(np.int32)


def _texel_dirs(H: int, W: int):
    th = (np.arange(H) + 0.5) / H * np.pi
    ph = (np.arange(W) + 0.5) / W * 2 * np.pi - np.pi
    th, ph = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(th) * np.sin(ph), np.cos(th), -np.sin(th) * np.cos(ph)], -1)


def env_uniform(value=1.0, H: int = 256, W: int = 512) -> EnvMap:
    v = np.broadcast_to(np.asarray(value, np.float32), (3,))
    return EnvMap(_f32(np.broadcast_to(v, (H, W, 3))))


def env_sky_sun(seed: int = 0, H: int = 256, W: int = 512, kappa: float = 300.0) -> EnvMap:
    """Sky gradient tinted per state plus a sun lobe of log-normal intensity."""
    rng = np.random.default_rng(10_000 + seed)
    w = _texel_dirs(H, W)
    tint = rng.uniform(0.7, 1.0, size=3)
    sky = (0.2 + 0.3 * np.maximum(0.0, w[..., 1:2])) * tint
    y = rng.uniform(0.25, 0.9)
    phi = rng.uniform(0, 2 * np.pi)
    sun = np.array([np.sqrt(1 - y * y) * np.cos(phi), y, np.sqrt(1 - y * y) * np.sin(phi)])
    intensity = np.exp(rng.normal(np.log(50.0), 0.5))
    lobe = intensity * np.exp(kappa * (w @ sun - 1.0))[..., None] * np.array([1.0, 0.95, 0.85])
    return EnvMap(_f32(sky + lobe))


def env_smooth(seed: int = 0, H: int = 64, W: int = 128) -> EnvMap:
    """Low-frequency positive environment (for quadrature checks)."""
    rng = np.random.default_rng(20_000 + seed)
    w = _texel_dirs(H, W)
    c = rng.uniform(-0.5, 0.5, size=(3, 3))
    base = 1.0 + 0.6 * np.tanh(w @ c)
    return EnvMap(_f32(np.clip(base, 0.2, None)))


def scene_with(scene: Scene, **kw) -> Scene:
    return replace(scene, **kw)
