"""Request server over several resident scenes (continuous batching; see grtx_server_* in
include/grtx.h). Argument marshalling only: admission, step scheduling and completion
tracking run in the library."""
from __future__ import annotations

import ctypes as C

import torch

from . import native as N
from .render import Scene, trace_params


class Server:
    def __init__(self, scenes: list[Scene], k=16, traversal="checkpoint", max_rays_per_step=0, max_inflight=0,
                 stream: torch.cuda.Stream | None = None, **params):
        self.scenes = list(scenes)
        self.stream = stream or torch.cuda.Stream()
        alpha_min = self.scenes[0].alpha_min
        self.params = trace_params(k=k, traversal=traversal, alpha_min=alpha_min, **params)
        arr = (C.c_void_p * len(self.scenes))(*[s.handle for s in self.scenes])
        out = C.c_void_p()
        N.check(N.lib().grtx_server_create(arr, len(self.scenes), C.byref(self.params), int(max_rays_per_step),
                                           int(max_inflight), C.c_void_p(self.stream.cuda_stream), C.byref(out)),
                "grtx_server_create")
        self.handle = out.value
        self._keep = {}

    def submit(self, requests):
        """requests: iterable of (scene_id, camera dict, rgbT output tensor [W*H, 4], tag)."""
        reqs = list(requests)
        arr = (N.grtx_request * len(reqs))()
        for i, (sid, cam, out, tag) in enumerate(reqs):
            arr[i].scene_id = int(sid)
            arr[i].cam = N.make_camera(cam)
            arr[i].d_rgbT = out.data_ptr()
            arr[i].tag = int(tag)
            self._keep[int(tag)] = out
        N.check(N.lib().grtx_server_submit(C.c_void_p(self.handle), arr, len(reqs)), "grtx_server_submit")

    def poll(self, wait=False, max_done=4096):
        done = (N.grtx_completion * max_done)()
        n = C.c_int(0)
        N.check(N.lib().grtx_server_poll(C.c_void_p(self.handle), done, max_done, C.byref(n), int(bool(wait))),
                "grtx_server_poll")
        res = []
        for i in range(n.value):
            c = done[i]
            self._keep.pop(int(c.tag), None)
            res.append(dict(tag=int(c.tag), status=int(c.status), t_admit=float(c.t_admit), t_done=float(c.t_done)))
        return res

    def load(self):
        a, b = C.c_int(0), C.c_int(0)
        N.check(N.lib().grtx_server_load(C.c_void_p(self.handle), C.byref(a), C.byref(b)), "grtx_server_load")
        return a.value, b.value

    def render_requests(self, requests):
        reqs = list(requests)
        arr = (N.grtx_request * len(reqs))()
        for i, (sid, cam, out, tag) in enumerate(reqs):
            arr[i].scene_id = int(sid)
            arr[i].cam = N.make_camera(cam)
            arr[i].d_rgbT = out.data_ptr()
            arr[i].tag = int(tag)
        done = (N.grtx_completion * max(len(reqs), 1))()
        n = C.c_int(0)
        N.check(N.lib().grtx_render_requests(C.c_void_p(self.handle), arr, len(reqs), done, C.byref(n), None),
                "grtx_render_requests")
        return [dict(tag=int(done[i].tag), status=int(done[i].status), t_admit=float(done[i].t_admit),
                     t_done=float(done[i].t_done)) for i in range(n.value)]

    def close(self):
        if getattr(self, "handle", None):
            N.lib().grtx_server_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
