"""B300-native differentiable ray tracing of 2D Gaussian surfels with
one-bounce physically based shading (LightFuse hot path).

All compute runs in the hand-written sm_103a kernels of liblightfuse.so
(C ABI in include/lightfuse.h); this package only marshals arguments.
"""
from . import _native  # noqa: F401
from .tracer import SceneTensors, Tracer, camera_struct, default_params, split_surfel_grad  # noqa: F401
from .render import StateRender, SurfelRender, render, render_state  # noqa: F401
from .checkpoint import Checkpoint, load_checkpoint, restore, save_checkpoint  # noqa: F401


def load_library():
    """Load liblightfuse.so (raises if the CUDA extension has not been built)."""
    return _native.load()
