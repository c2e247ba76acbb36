"""Served edit-and-render loop (lf_serve_*) and the plain per-request loop it
is compared with.  Marshalling and request timing only; the work runs in the
library (scheduler thread, edits, batched kernels)."""
from __future__ import annotations

import ctypes as C
import queue
import threading
import time
from typing import Optional

import numpy as np
import torch

from . import _native as N
from .tracer import Tracer, camera_struct

KIND = dict(none=0, move=1, material=2, env=3)


def request_struct(edit: Optional[dict], cam, spp: int, seed: int) -> N.LfRequest:
    r = N.LfRequest()
    e = edit or dict(kind="none")
    r.edit.kind = KIND[e["kind"]]
    if e["kind"] in ("move", "material"):
        r.edit.object_id = int(e["object"])
    if e["kind"] == "move":
        r.edit.R[:] = [float(v) for v in np.asarray(e["R"], np.float32).reshape(-1)]
        r.edit.t[:] = [float(v) for v in np.asarray(e["t"], np.float32).reshape(-1)]
    if e["kind"] == "material":
        if e.get("albedo") is not None:
            r.edit.albedo[:] = [float(v) for v in e["albedo"]]
            r.edit.set_albedo = 1
        r.edit.metallic = float(e.get("metallic", -1.0))
        r.edit.roughness = float(e.get("roughness", -1.0))
    else:
        r.edit.metallic = -1.0
        r.edit.roughness = -1.0
    if e["kind"] == "env":
        r.edit.env_id = int(e["env"])
    r.cam = camera_struct(cam)
    r.spp = int(spp)
    r.seed = int(seed)
    return r


class Server:
    """lf_serve: continuous batching over a device-resident scene."""

    def __init__(self, tracer: Tracer, budget_bytes: int, max_slots: int = 8, n_streams: int = 4,
                 batch_window_us: int = 0):
        self.tr = tracer
        self.lib = tracer.lib
        h = C.c_void_p()
        st = self.lib.lf_serve_create(tracer.ctx, C.c_size_t(int(budget_bytes)), int(max_slots), int(n_streams),
                                      int(batch_window_us), C.byref(h))
        if st != N.LF_OK:
            raise N.LightFuseError(st, "lf_serve_create")
        self.h = h

    def submit(self, edit, cam, spp, seed) -> int:
        r = request_struct(edit, cam, spp, seed)
        t = C.c_uint64()
        st = self.lib.lf_serve_submit(self.h, C.byref(r), C.byref(t))
        if st != N.LF_OK:
            raise N.LightFuseError(st, "lf_serve_submit")
        return t.value

    def cancel(self, ticket: int) -> int:
        """LF_OK when the request had not been admitted (its poll then returns
        LF_ERR_CANCELLED), LF_ERR_BUSY when it is already running or done."""
        return self.lib.lf_serve_cancel(self.h, C.c_uint64(ticket))

    def wait(self, ticket: int, timeout_ms: int = 600_000) -> int:
        return self.lib.lf_serve_wait(self.h, C.c_uint64(ticket), int(timeout_ms))

    def result(self, ticket: int, cam, want_frame: bool = True):
        """(status, frame (H, W, 3) or None, timing dict); call after wait()."""
        done = C.c_int()
        frame = np.empty((cam.height, cam.width, 3), np.float32) if want_frame else None
        tm = N.LfTiming()
        st = self.lib.lf_serve_poll(self.h, C.c_uint64(ticket), C.byref(done),
                                    frame.ctypes.data_as(C.c_void_p) if want_frame else None,
                                    frame.size if want_frame else 0, C.byref(tm))
        timing = dict(t_submit=tm.t_submit, t_admit=tm.t_admit, t_start=tm.t_start, t_done=tm.t_done, rays=tm.rays)
        return st, (frame if st == N.LF_OK else None), timing

    def close(self):
        if getattr(self, "h", None):
            self.lib.lf_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_served(server: Server, requests, keep_frames: bool = False, timeout_ms: int = 120_000):
    """Submit at the requests' arrival times from one thread while this thread
    collects results as they finish (a finished request holds one of the
    server's pinned frames until it is collected).  Returns per-request
    records; status LF_ERR_TIMEOUT for one not finished within timeout_ms."""
    t0 = time.perf_counter()
    submitted: "queue.Queue" = queue.Queue()

    def submitter():
        for i, rq in enumerate(requests):
            delay = t0 + rq.arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            try:
                submitted.put(server.submit(rq.edit, rq.cam, rq.spp, rq.seed))
            except Exception as exc:  # hand the failure to the collector
                submitted.put(exc)

    th = threading.Thread(target=submitter)
    th.start()
    out = []
    try:
        for rq in requests:
            ticket = submitted.get()
            if isinstance(ticket, Exception):
                raise ticket
            if server.wait(ticket, timeout_ms) != N.LF_OK:
                out.append(dict(status=N.LF_ERR_TIMEOUT, frame=None, latency=float("nan")))
                continue
            st, frame, tm = server.result(ticket, rq.cam, want_frame=keep_frames)
            out.append(dict(status=st, frame=frame, latency=tm["t_done"] - tm["t_submit"], **tm))
    finally:
        th.join()
    return out


def apply_edit(tracer: Tracer, edit, env_state: dict):
    if edit is None or edit["kind"] == "none":
        return
    if edit["kind"] == "move":
        tracer.refit(edit["object"], edit["R"], edit["t"])
    elif edit["kind"] == "material":
        tracer.set_material(edit["object"], edit.get("albedo"), edit.get("metallic", -1.0),
                            edit.get("roughness", -1.0))
    elif edit["kind"] == "env":
        env_state["env"] = edit["env"]


def run_plain(tracer: Tracer, requests, keep_frames: bool = False, env0: int = 0):
    """The plain per-request loop: apply the edit, rebuild every BVH from
    scratch, render, copy the frame to the host, synchronise; FIFO."""
    t0 = time.perf_counter()
    env_state = dict(env=env0)
    out = []
    for rq in requests:
        arrival = t0 + rq.arrival
        now = time.perf_counter()
        if now < arrival:
            time.sleep(arrival - now)
        apply_edit(tracer, rq.edit, env_state)
        tracer.build(tracer.scene)
        g = tracer.trace_primary(rq.cam, env_state["env"])
        rgb = tracer.shade(rq.cam, g, env_state["env"], rq.spp, rq.seed)
        frame = rgb.cpu().numpy()
        tracer.sync()
        done = time.perf_counter()
        out.append(dict(status=0, frame=frame if keep_frames else None, latency=done - arrival,
                        t_submit=arrival, t_done=done))
    return out
