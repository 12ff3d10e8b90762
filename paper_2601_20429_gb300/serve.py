"""Request server over several resident scenes (continuous batching; see grtx_server_* in
include/grtx.h). Argument marshalling only: admission, step scheduling and completion
tracking run in the library."""
from __future__ import annotations

import atexit
import ctypes as C
import weakref

import torch

from . import native as N
from .render import Scene, trace_params


# servers still open when the interpreter exits are closed first (each runs a native scheduler
# thread, which must stop before the CUDA runtime is torn down)
_open_servers: "weakref.WeakSet[Server]" = weakref.WeakSet()


@atexit.register
def _close_open_servers():
    for srv in list(_open_servers):
        try:
            srv.close()
        except Exception:
            pass


class Server:
    def __init__(self, scenes: list[Scene], k=16, traversal="checkpoint", max_rays_per_step=0, max_inflight=0,
                 stream: torch.cuda.Stream | None = None, mem_budget_bytes=0, linger_us: float | None = None,
                 size_ns_per_ray: float | None = None, append_guard: bool = True, **params):
        self.scenes = list(scenes)
        self.stream = stream or torch.cuda.Stream()
        alpha_min = self.scenes[0].alpha_min
        self.params = trace_params(k=k, traversal=traversal, alpha_min=alpha_min, **params)
        arr = (C.c_void_p * len(self.scenes))(*[s.handle for s in self.scenes])
        out = C.c_void_p()
        N.check(N.lib().grtx_server_create(arr, len(self.scenes), C.byref(self.params), int(mem_budget_bytes),
                                           int(max_rays_per_step), int(max_inflight),
                                           C.c_void_p(self.stream.cuda_stream), C.byref(out)),
                "grtx_server_create")
        self.handle = out.value
        _open_servers.add(self)
        if linger_us is not None:
            N.check(N.lib().grtx_server_set_linger(C.c_void_p(self.handle), int(round(linger_us * 1000))),
                    "grtx_server_set_linger")
        if not append_guard:
            N.check(N.lib().grtx_server_set_append_guard(C.c_void_p(self.handle), 0), "grtx_server_set_append_guard")
        if size_ns_per_ray is not None:
            N.check(N.lib().grtx_server_set_order(C.c_void_p(self.handle), float(size_ns_per_ray)),
                    "grtx_server_set_order")
        self._keep = {}
        self._shape = {}

    def submit(self, requests):
        """requests: iterable of (scene_id, camera dict, rgbT output tensor [W*H, 4] or None, tag).
        With None the server allocates the output from its memory budget when it admits the
        request; poll() then returns it as a tensor view ("rgbT"), valid until release()."""
        reqs = list(requests)
        arr = (N.grtx_request * len(reqs))()
        for i, (sid, cam, out, tag) in enumerate(reqs):
            arr[i].scene_id = int(sid)
            arr[i].cam = N.make_camera(cam)
            arr[i].d_rgbT = out.data_ptr() if out is not None else None
            arr[i].tag = int(tag)
        N.check(N.lib().grtx_server_submit(C.c_void_p(self.handle), arr, len(reqs)), "grtx_server_submit")
        for sid, cam, out, tag in reqs:
            self._keep[int(tag)] = out
            self._shape[int(tag)] = int(cam["width"]) * int(cam["height"])

    def _completion(self, c):
        tag = int(c.tag)
        own = self._keep.pop(tag, None)
        n = self._shape.pop(tag, 0)
        res = dict(tag=tag, status=int(c.status), t_admit=float(c.t_admit), t_done=float(c.t_done),
                   d_rgbT=int(c.d_rgbT or 0))
        if own is None and c.d_rgbT:
            res["rgbT"] = N.device_view(int(c.d_rgbT), (n, 4))
        return res

    def poll(self, wait=False, max_done=4096):
        done = (N.grtx_completion * max_done)()
        n = C.c_int(0)
        N.check(N.lib().grtx_server_poll(C.c_void_p(self.handle), done, max_done, C.byref(n), int(bool(wait))),
                "grtx_server_poll")
        return [self._completion(done[i]) for i in range(n.value)]

    def release(self, completion):
        """Give a server-owned output back (once every read of it has completed)."""
        ptr = completion["d_rgbT"] if isinstance(completion, dict) else int(completion)
        N.check(N.lib().grtx_server_release(C.c_void_p(self.handle), C.c_void_p(ptr)), "grtx_server_release")

    def info(self) -> dict:
        i = N.grtx_server_info()
        N.check(N.lib().grtx_server_get_info(C.c_void_p(self.handle), C.byref(i)), "grtx_server_get_info")
        return {name: int(getattr(i, name)) for name, _ in N.grtx_server_info._fields_}

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
                     t_done=float(done[i].t_done), d_rgbT=int(done[i].d_rgbT or 0)) for i in range(n.value)]

    def close(self):
        if getattr(self, "handle", None):
            N.lib().grtx_server_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
