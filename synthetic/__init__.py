"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package draws scenes, environment maps, cameras and pixel subsets.  It
holds none of the tracing or shading arithmetic: every array it returns is
plain input data (float32), and both sides consume the same arrays.
"""
from .scenes import (  # noqa: F401
    Scene, Camera, EnvMap,
    random_surfels, box_shell, object_surfels, scene_c1, scene_c2, scene_c3_subset,
    scene_c4, env_uniform, env_sky_sun, camera_c1, camera_c2, camera_c4,
    pixel_subset, perturb_scene, rigid_motion, quat_to_axes,
)
