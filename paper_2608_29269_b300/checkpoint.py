"""Scene checkpoints: everything a render, a served scene or an inverse-rendering
run needs to resume, in one ``.npz`` file.

Saved: the surfel attributes (Eq. 1) and the object layout, the environment
maps by slot, the method constants (``lf_params``), named per-state object
transforms (Eq. 2: ``R`` (M, 3, 3) and ``t`` (M, 3) for objects 1..M) and the
forward seed and spp that the path-replay adjoint replays (Sec. 3.3).  Not
saved: the BVH and the environment sampling tables.  `restore` rebuilds them
through ``lf_bvh_build`` / ``lf_env_set``, which takes milliseconds and keeps
the file independent of the library's internal node layout.

Host-side marshalling only (numpy / torch); nothing here computes.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Dict, Optional, Tuple

import numpy as np
import torch

from . import _native as N
from .tracer import SCENE_FIELDS, SceneTensors

FORMAT_VERSION = 1


@dataclass
class Checkpoint:
    scene: SceneTensors
    envs: Dict[int, torch.Tensor] = field(default_factory=dict)
    params: Dict[str, float] = field(default_factory=dict)  # lf_params fields
    states: Dict[str, Tuple[np.ndarray, np.ndarray]] = field(default_factory=dict)
    seed: Optional[int] = None
    spp: Optional[int] = None

    def lf_params(self) -> N.LfParams:
        """The saved constants as an lf_params struct (fields not saved keep 0)."""
        p = N.LfParams()
        for k, v in self.params.items():
            setattr(p, k, v)
        return p


def _params_dict(params) -> Dict[str, float]:
    if params is None:
        return {}
    if isinstance(params, dict):
        return dict(params)
    return {name: getattr(params, name) for name, _ in params._fields_}


def save_checkpoint(path, scene: SceneTensors, envs: Optional[Dict[int, torch.Tensor]] = None, params=None,
                    states: Optional[Dict[str, Tuple[np.ndarray, np.ndarray]]] = None, seed: Optional[int] = None,
                    spp: Optional[int] = None) -> None:
    """Write one .npz: scene tensors (any device), env maps {slot: (H, W, 3)},
    params (an LfParams or a dict), states {name: (R, t)}, seed, spp."""
    arrays = {"version": np.array(FORMAT_VERSION, np.int32),
              "object_offsets": np.asarray(list(scene.object_offsets) or [0, scene.n], np.int32)}
    for k in SCENE_FIELDS:
        arrays["scene_" + k] = getattr(scene, k).detach().cpu().numpy().astype(np.float32)
    for slot, rgb in (envs or {}).items():
        if not 0 <= int(slot) < 16:
            raise ValueError(f"environment slot {slot} outside 0..15")
        arrays[f"env_{int(slot)}"] = torch.as_tensor(rgb).detach().cpu().numpy().astype(np.float32)
    pd = _params_dict(params)
    arrays["param_names"] = np.array(sorted(pd), dtype="U32")
    arrays["param_values"] = np.array([float(pd[k]) for k in sorted(pd)], np.float64)
    names = sorted(states or {})
    arrays["state_names"] = np.array(names, dtype="U64")
    for i, name in enumerate(names):
        R, t = states[name]
        arrays[f"state_{i}_R"] = np.asarray(R, np.float32).reshape(-1, 3, 3)
        arrays[f"state_{i}_t"] = np.asarray(t, np.float32).reshape(-1, 3)
    arrays["seed"] = np.array(-1 if seed is None else int(seed), np.int64)
    arrays["spp"] = np.array(-1 if spp is None else int(spp), np.int64)
    with open(path, "wb") as f:
        np.savez(f, **arrays)


def load_checkpoint(path, device="cuda") -> Checkpoint:
    """Read a checkpoint written by `save_checkpoint`; tensors land on `device`."""
    with np.load(path, allow_pickle=False) as z:
        version = int(z["version"])
        if version != FORMAT_VERSION:
            raise ValueError(f"checkpoint format {version}, expected {FORMAT_VERSION}")
        kw = {k: torch.as_tensor(z["scene_" + k], device=device).contiguous() for k in SCENE_FIELDS}
        scene = SceneTensors(**kw, object_offsets=[int(v) for v in z["object_offsets"]])
        envs = {int(k[4:]): torch.as_tensor(z[k], device=device).contiguous() for k in z.files if k.startswith("env_")}
        params = {}
        int_fields = {name for name, ty in N.LfParams._fields_ if ty is C.c_int}
        for name, value in zip(z["param_names"], z["param_values"]):
            params[str(name)] = int(value) if str(name) in int_fields else float(value)
        states = {str(name): (z[f"state_{i}_R"].copy(), z[f"state_{i}_t"].copy())
                  for i, name in enumerate(z["state_names"])}
        seed, spp = int(z["seed"]), int(z["spp"])
    n = scene.n
    offs = scene.object_offsets
    if offs[0] != 0 or offs[-1] != n or any(b < a for a, b in zip(offs, offs[1:])):
        raise ValueError("checkpoint object offsets do not partition the surfels")
    return Checkpoint(scene=scene, envs=envs, params=params, states=states, seed=None if seed < 0 else seed,
                      spp=None if spp < 0 else spp)


def restore(tracer, ckpt: Checkpoint) -> None:
    """Rebuild the BVH of the checkpoint's scene and register its environment
    maps on `tracer` (the scene tensors must be on the tracer's device)."""
    tracer.build(ckpt.scene)
    for slot, rgb in sorted(ckpt.envs.items()):
        tracer.set_env(slot, rgb)
