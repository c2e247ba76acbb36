"""Seeded request streams for the served edit-and-render loop.

Each request is an edit (rigid move of an object, material edit or
environment swap) plus a camera at its own resolution and sample count,
arriving as a Poisson process.  Pure input data: no rendering here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .scenes import Camera, rigid_motion


@dataclass
class Request:
    arrival: float          # seconds after the start of the stream
    edit: dict              # {"kind": "move"|"material"|"env"|"none", ...}
    cam: Camera
    spp: int
    seed: int


def request_stream(n, rate, scene, n_envs=3, resolutions=(256, 512, 800, 1024), spps=(4, 8, 16, 32),
                   cam_fn=None, seed=0):
    """n requests with exponential inter-arrival times (mean 1/rate s)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    n_obj = scene.n_objects
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        kind = ["move", "material", "env"][int(rng.integers(0, 3))]
        if kind == "move":
            k = int(rng.integers(1, n_obj))
            lo, hi = scene.object_offsets[k], scene.object_offsets[k + 1]
            R, tr = rigid_motion(rng, scene.mu[lo:hi].mean(0), max_shift=0.1)
            edit = dict(kind="move", object=k, R=R, t=tr)
        elif kind == "material":
            k = int(rng.integers(1, n_obj))
            edit = dict(kind="material", object=k, albedo=rng.uniform(0, 1, 3).astype(np.float32),
                        metallic=float(rng.uniform(0, 1)), roughness=float(rng.uniform(0.05, 1)))
        else:
            edit = dict(kind="env", env=int(rng.integers(0, n_envs)))
        res = int(resolutions[int(rng.integers(0, len(resolutions)))])
        cam = cam_fn(res) if cam_fn else Camera((0.0, -0.2, 1.9), (0.0, -1.5, -0.2), (0.0, 1.0, 0.0), 60.0, res, res)
        out.append(Request(t, edit, cam, int(spps[int(rng.integers(0, len(spps)))]), int(rng.integers(0, 2**31))))
    return out
