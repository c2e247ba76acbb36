"""ctypes declarations of the C ABI in include/lightfuse.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblightfuse.so")

LF_OK, LF_ERR_INVALID, LF_ERR_OOM, LF_ERR_CUDA, LF_ERR_STACK, LF_ERR_ROUND_LIMIT, LF_ERR_TIMEOUT, LF_ERR_BUSY, \
    LF_ERR_NOT_BUILT, LF_ERR_BOUNDS, LF_ERR_CANCELLED = range(11)
STATUS_NAMES = ["LF_OK", "LF_ERR_INVALID", "LF_ERR_OOM", "LF_ERR_CUDA", "LF_ERR_STACK", "LF_ERR_ROUND_LIMIT",
                "LF_ERR_TIMEOUT", "LF_ERR_BUSY", "LF_ERR_NOT_BUILT", "LF_ERR_BOUNDS", "LF_ERR_CANCELLED"]

LF_MAX_OBJECTS = 64
LF_MAX_ENVS = 16
LF_KBUF = 32
LF_GBUF_CHANNELS = 32
LF_GBUF_DIFF = 17
CH = dict(T=0, W=1, depth=2, x=3, n=6, a=9, m=12, r=13, rho=14, nlen=17, hits=18, t_stop=19, id_stop=20, dir=21,
          stopkey_lo=24, x_lo=25, n_lo=28, r_lo=31)
G_STRIDE = 17


class LfParams(C.Structure):
    _fields_ = [("T_min", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("support_r2", C.c_float),
                ("eps_w", C.c_float), ("t_min", C.c_float), ("ray_offset", C.c_float), ("p_spec", C.c_float),
                ("max_rounds", C.c_int), ("brdf_mode", C.c_int), ("sampling_mode", C.c_int), ("sampler", C.c_int)]


class LfScene(C.Structure):
    _fields_ = [("mu_dev", C.c_void_p), ("tu_dev", C.c_void_p), ("tv_dev", C.c_void_p), ("scale_dev", C.c_void_p),
                ("opacity_dev", C.c_void_p), ("albedo_dev", C.c_void_p), ("metallic_dev", C.c_void_p),
                ("roughness_dev", C.c_void_p), ("n", C.c_int), ("object_offsets", C.POINTER(C.c_int)),
                ("n_objects", C.c_int)]


class LfCamera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3), ("fovy_deg", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class LfEdit(C.Structure):
    _fields_ = [("kind", C.c_int), ("object_id", C.c_int), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("albedo", C.c_float * 3), ("metallic", C.c_float), ("roughness", C.c_float),
                ("set_albedo", C.c_int), ("env_id", C.c_int)]


class LfRequest(C.Structure):
    _fields_ = [("edit", LfEdit), ("cam", LfCamera), ("spp", C.c_int), ("seed", C.c_uint64)]


class LfTiming(C.Structure):
    _fields_ = [("t_submit", C.c_double), ("t_admit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("rays", C.c_ulonglong)]


# (name, restype, argtypes) for every exported symbol of include/lightfuse.h
_P = C.c_void_p
SIGNATURES = [
    ("lf_params_default", C.c_int, [C.POINTER(LfParams)]),
    ("lf_create", C.c_int, [C.POINTER(LfParams), _P, C.POINTER(_P)]),
    ("lf_destroy", C.c_int, [_P]),
    ("lf_set_stream", C.c_int, [_P, _P]),
    ("lf_last_error", C.c_char_p, [_P]),
    ("lf_sync", C.c_int, [_P]),
    ("lf_bvh_build", C.c_int, [_P, C.POINTER(LfScene)]),
    ("lf_bvh_refit", C.c_int, [_P, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    ("lf_scene_sync", C.c_int, [_P, C.c_int]),
    ("lf_material_set", C.c_int, [_P, C.c_int, C.POINTER(C.c_float), C.c_float, C.c_float]),
    ("lf_state_assemble", C.c_int, [_P, C.POINTER(LfScene), C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    ("lf_state_pullback", C.c_int, [_P, C.POINTER(C.c_float), _P, _P]),
    ("lf_env_set", C.c_int, [_P, C.c_int, _P, C.c_int, C.c_int]),
    ("lf_trace_primary", C.c_int, [_P, C.POINTER(LfCamera), C.c_int, _P]),
    ("lf_shade_scratch_bytes", C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    ("lf_shade_bounce", C.c_int, [_P, C.POINTER(LfCamera), _P, C.c_int, C.c_int, C.c_uint64, _P, _P, _P,
                                  C.c_size_t]),
    ("lf_shade_bounce_static", C.c_int, [_P, C.POINTER(LfCamera), _P, C.c_int, C.c_int, C.c_uint64, _P, _P]),
    ("lf_shade_sample_terms", C.c_int, [_P, C.POINTER(LfCamera), _P, C.c_int, C.c_int, _P, C.c_size_t, _P]),
    ("lf_backward_scratch_bytes", C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    ("lf_trace_backward", C.c_int, [_P, C.POINTER(LfCamera), _P, C.c_int, C.c_int, C.c_uint64, _P, _P, _P, _P, _P,
                                    _P, C.c_size_t]),
    ("lf_set_counters", C.c_int, [_P, _P]),
    ("lf_profile", C.c_int, [_P, C.c_int]),
    ("lf_profile_read", C.c_int, [_P, C.POINTER(C.c_float)]),
    ("lf_philox", C.c_int, [_P, _P, C.c_int, C.c_uint32, C.c_uint32, _P]),
    ("lf_measure_l2_read", C.c_int, [_P, C.c_size_t, C.c_int, C.POINTER(C.c_float)]),
    ("lf_opacity_loss", C.c_int, [_P, C.POINTER(LfCamera), _P, C.c_float, _P, C.POINTER(C.c_double)]),
    ("lf_scale_loss", C.c_int, [_P, _P, C.c_int, C.c_float, C.c_float, _P, C.POINTER(C.c_double)]),
    ("lf_env_tv_loss", C.c_int, [_P, _P, C.c_int, C.c_int, C.c_float, _P, C.POINTER(C.c_double)]),
    ("lf_geometry_loss_scratch_bytes", C.c_size_t, [C.c_int, C.c_int]),
    ("lf_geometry_loss", C.c_int, [_P, C.POINTER(LfCamera), _P, _P, _P, _P, C.c_float, C.POINTER(C.c_float), _P, _P,
                                   C.c_size_t, C.POINTER(C.c_double)]),
    ("lf_env_tables", C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    ("lf_bvh_info", C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("lf_bvh_wide_node_bytes", C.c_int, []),
    ("lf_bvh_copy_wide", C.c_int, [_P, C.c_int, _P, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("lf_bvh_copy_nodes", C.c_int, [_P, C.c_int, _P, C.c_size_t]),
    ("lf_serve_create", C.c_int, [_P, C.c_size_t, C.c_int, C.c_int, C.c_int, C.POINTER(_P)]),
    ("lf_serve_submit", C.c_int, [_P, C.POINTER(LfRequest), C.POINTER(C.c_uint64)]),
    ("lf_serve_poll", C.c_int, [_P, C.c_uint64, C.POINTER(C.c_int), _P, C.c_size_t, C.POINTER(LfTiming)]),
    ("lf_serve_wait", C.c_int, [_P, C.c_uint64, C.c_int]),
    ("lf_serve_cancel", C.c_int, [_P, C.c_uint64]),
    ("lf_serve_destroy", C.c_int, [_P]),
]

_lib = None


def load(path: str = None):
    """Load liblightfuse.so; fails loudly when the CUDA extension is missing.
    LIGHTFUSE_LIB, when set, names another build of the same sources to load
    (the bounds-checked one, for instance)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("LIGHTFUSE_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA extension not built: {path} is missing (run paper_2608_29269_b300/build.py)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LightFuseError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
