"""lf_shade_bounce_static: shading for callers that cannot allocate device memory.

Such callers (a host whose device memory belongs to another allocator, a
plugin that may not call cudaMalloc, a render loop that must not allocate
after start-up) cannot hand lf_shade_bounce its per-sample scratch buffer;
this entry point uses a fixed array inside the library instead.  The test
calls it through the C ABI twice in a row and compares each image with the
existing entry point's on the same inputs, checks that those two calls left
the device's free memory and torch's allocation unchanged (nothing was
allocated), and that a request larger than the array is refused.  This file
is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from synthetic import scenes as S

pytestmark = pytest.mark.gpu
TOL = 1e-4  # the radiance tolerance of the parity tests


def test_static_scratch_shading_matches_caller_scratch_twice():
    import torch
    from paper_2608_29269_b300 import SceneTensors, Tracer, camera_struct
    from paper_2608_29269_b300 import _native as N
    from paper_2608_29269_b300.build import build
    build()
    lib = N.load()
    sc = S.random_surfels(2000, seed=3)
    cam = S.Camera((0.0, 0.0, 2.5), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, 96, 80)
    spp = 6
    tr = Tracer()
    tr.build(SceneTensors.from_numpy(sc))
    tr.set_env(0, torch.as_tensor(S.env_sky_sun(4).rgb, device="cuda"))
    g = tr.trace_primary(cam, 0)
    ref = tr.shade(cam, g, 0, spp=spp, seed=99)
    tr.sync()
    c = camera_struct(cam)

    def call(out):
        st = lib.lf_shade_bounce_static(tr.ctx, C.byref(c), C.c_void_p(g.data_ptr()), 0, spp, C.c_uint64(99),
                                        C.c_void_p(out.data_ptr()), None)
        assert st == N.LF_OK, lib.lf_last_error(tr.ctx)

    # outputs are allocated up front; a first call outside the measured span
    outs = [torch.full_like(ref, float("nan")) for _ in range(2)]
    call(torch.empty_like(ref))
    tr.sync()
    torch.cuda.synchronize()
    free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for out in outs:
        call(out)
        tr.sync()
    torch.cuda.synchronize()
    free1, torch1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert free1 == free0, (free0, free1)
    assert torch1 == torch0, (torch0, torch1)
    for out in outs:
        diff = (out - ref).abs().max().item()
        assert diff <= TOL, diff
    # a request beyond the array's capacity is refused before anything runs
    big = S.Camera((0.0, 0.0, 2.5), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, 512, 512)
    cb = camera_struct(big)
    out = torch.empty((512, 512, 3), device="cuda")
    gb = torch.zeros((N.LF_GBUF_CHANNELS, 512, 512), device="cuda")
    st = lib.lf_shade_bounce_static(tr.ctx, C.byref(cb), C.c_void_p(gb.data_ptr()), 0, 2, C.c_uint64(1),
                                    C.c_void_p(out.data_ptr()), None)
    assert st == N.LF_ERR_INVALID
    assert b"exceeds the static scratch capacity" in lib.lf_last_error(tr.ctx)
    tr.sync()
