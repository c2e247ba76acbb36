"""Served edit-and-render loop: each frame is the same alone and in the mix,
equals the plain per-request rebuild-and-render loop, and admission respects
the memory budget; malformed requests are refused."""
import dataclasses

import numpy as np
import pytest

from synthetic import scenes as S
from synthetic.requests import request_stream
from tests._helpers import gpu_tracer

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _setup():
    sc = S.scene_c2(0, per_face=3000, per_object=8000)
    tr, st = gpu_tracer(sc, [S.env_sky_sun(i, 64, 128) for i in range(3)])
    return sc, tr, st


def _requests(sc, n=14, seed=3):
    cam_fn = lambda res: S.Camera((0.0, -0.5, 1.8), (0.0, -1.5, 0.0), (0.0, 1.0, 0.0), 60.0, res, res)
    reqs = request_stream(n, rate=1000.0, scene=sc, n_envs=3, resolutions=(48, 64, 96), spps=(2, 3, 4),
                          cam_fn=cam_fn, seed=seed)
    return [dataclasses.replace(r, arrival=0.0) for r in reqs]  # a burst: requests share launches


def test_served_frames_equal_alone_and_plain_loop():
    from paper_2608_29269_b300.serve import Server, run_plain, run_served
    sc, tr, st = _setup()
    reqs = _requests(sc)
    srv = Server(tr, budget_bytes=2 << 30, max_slots=8, n_streams=3, batch_window_us=50_000)
    mix = run_served(srv, reqs, keep_frames=True)
    srv.close()
    srv1 = Server(tr, budget_bytes=2 << 30, max_slots=1, n_streams=1)
    alone = []
    for rq in reqs:  # one request at a time
        alone += run_served(srv1, [rq], keep_frames=True)
    srv1.close()
    plain = run_plain(tr, reqs, keep_frames=True)  # mutates the tracer's scene: last
    batched = len({round(r["t_start"], 9) for r in mix}) < len(mix)
    assert batched, "no two requests shared a launch group"
    for i, (a, b, c) in enumerate(zip(mix, alone, plain)):
        assert a["status"] == 0 and b["status"] == 0, (i, a["status"], b["status"])
        assert a["t_submit"] <= a["t_admit"] <= a["t_start"] <= a["t_done"]
        assert np.abs(a["frame"] - b["frame"]).max() <= TOL, i
        assert np.abs(a["frame"] - c["frame"]).max() <= TOL, i
        assert np.isfinite(a["frame"]).all() and a["frame"].mean() > 0


def test_admission_budget_and_malformed_requests():
    from paper_2608_29269_b300 import _native as N
    from paper_2608_29269_b300.serve import Server
    sc, tr, st = _setup()
    cam = S.Camera((0.0, -0.5, 1.8), (0.0, -1.5, 0.0), (0.0, 1.0, 0.0), 60.0, 96, 96)
    srv = Server(tr, budget_bytes=1 << 20, max_slots=2, n_streams=1)  # 1 MiB: too small for any frame
    t = srv.submit(None, cam, 4, 1)
    assert srv.wait(t, 60_000) == N.LF_OK
    stt, frame, _ = srv.result(t, cam)
    assert stt == N.LF_ERR_OOM and frame is None
    with pytest.raises(N.LightFuseError):
        srv.submit(dict(kind="move", object=99, R=np.eye(3), t=np.zeros(3)), cam, 4, 1)
    with pytest.raises(N.LightFuseError):
        srv.submit(dict(kind="move", object=1, R=2 * np.eye(3), t=np.zeros(3)), cam, 4, 1)
    with pytest.raises(N.LightFuseError):
        srv.submit(None, S.Camera((0, 0, 3), (0, 0, 0), (0, 1, 0), 60.0, 2048, 2048), 4, 1)
    with pytest.raises(N.LightFuseError):
        srv.submit(dict(kind="env", env=7), cam, 4, 1)
    srv.close()
    # a budget that fits one request at a time still serves every request
    srv = Server(tr, budget_bytes=24 << 20, max_slots=8, n_streams=2)
    ts = [srv.submit(None, cam, 4, k) for k in range(5)]
    for k in ts:
        assert srv.wait(k, 60_000) == N.LF_OK
        stt, frame, tm = srv.result(k, cam)
        assert stt == N.LF_OK and frame is not None
    srv.close()


def test_more_finished_requests_than_frames_keep_admission_going():
    """Every request of a burst larger than the pinned frame pool (2 x
    max_slots) completes when the client polls in order: the worker sleeps
    while the pool is empty and wakes when a poll hands a frame back."""
    import time
    from paper_2608_29269_b300 import _native as N
    from paper_2608_29269_b300.serve import Server
    sc, tr, st = _setup()
    cam = S.Camera((0.0, -0.5, 1.8), (0.0, -1.5, 0.0), (0.0, 1.0, 0.0), 60.0, 32, 32)
    srv = Server(tr, budget_bytes=1 << 30, max_slots=2, n_streams=2)  # 4 frames
    ts = [srv.submit(None, cam, 2, k) for k in range(11)]
    t0 = time.perf_counter()
    for k in ts:
        assert srv.wait(k, 30_000) == N.LF_OK
        stt, frame, _ = srv.result(k, cam)
        assert stt == N.LF_OK and frame is not None and np.isfinite(frame).all()
    assert time.perf_counter() - t0 < 30.0
    srv.close()


def test_pending_requests_can_be_cancelled():
    """A request withdrawn before admission finishes as LF_ERR_CANCELLED with
    no frame; one already admitted runs to the end; the server goes on."""
    from paper_2608_29269_b300 import _native as N
    from paper_2608_29269_b300.serve import Server
    sc, tr, st = _setup()
    cam = S.Camera((0.0, -0.5, 1.8), (0.0, -1.5, 0.0), (0.0, 1.0, 0.0), 60.0, 96, 96)
    srv = Server(tr, budget_bytes=2 << 30, max_slots=1, n_streams=1)
    tickets = [srv.submit(None, cam, 8, s) for s in range(6)]
    codes = [srv.cancel(t) for t in tickets[::-1]]  # the tail of a one-slot queue is still pending
    assert codes[0] == N.LF_OK
    assert srv.cancel(tickets[-1]) == N.LF_ERR_BUSY  # already done (cancelled)
    assert srv.cancel(10 ** 9) == N.LF_ERR_INVALID
    for t, c in zip(tickets[::-1], codes):
        assert c in (N.LF_OK, N.LF_ERR_BUSY)
        assert srv.wait(t, 60_000) == N.LF_OK
        status, frame, tm = srv.result(t, cam)
        if c == N.LF_OK:
            assert status == N.LF_ERR_CANCELLED and frame is None and tm["rays"] == 0
        else:
            assert status == N.LF_OK and np.isfinite(frame).all()
    t = srv.submit(None, cam, 4, 9)
    assert srv.wait(t, 60_000) == N.LF_OK and srv.result(t, cam)[0] == N.LF_OK
    srv.close()
