"""Build and load libgrtx.so (the CUDA C-ABI library) and expose its entry points.

This module is argument marshalling only: every step of rendering runs in the library's
kernels. Device memory and streams come from PyTorch tensors and streams; the functions take
tensors, pass their data pointers, and raise GrtxError on a non-zero status. Loading fails
loudly when the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import glob
import os
import subprocess
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(_PKG, "libgrtx.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lock = threading.Lock()
_lib = None


class GrtxError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what} failed: status {status} ({_status_text(status)}){': ' + detail if detail else ''}")


def _sources():
    return sorted(glob.glob(os.path.join(_CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(_CSRC, "*.cuh")) + glob.glob(os.path.join(_CSRC, "*.h")) +
            glob.glob(os.path.join(_INCLUDE, "*.h")))


def needs_build() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ for sm_103a (in parallel) and link libgrtx.so in-tree."""
    if not force and not needs_build():
        return LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I" + _INCLUDE, "-Xcompiler", "-fPIC,-fvisibility=hidden",
                    "-Xptxas", "-v"]
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(_BUILD, os.path.basename(src)[:-3] + ".o")
        log = open(obj + ".log", "w")
        procs.append((src, subprocess.Popen([NVCC] + flags + ["-c", src, "-o", obj], stdout=log,
                                            stderr=subprocess.STDOUT), log))
        objs.append(obj)
    failed = []
    for src, p, log in procs:
        p.wait()
        log.close()
        if p.returncode != 0:
            failed.append(src)
    if failed:
        msgs = []
        for src in failed:
            msgs.append(open(os.path.join(_BUILD, os.path.basename(src)[:-3] + ".o.log")).read()[-3000:])
        raise RuntimeError("nvcc failed for " + ", ".join(failed) + "\n" + "\n".join(msgs))
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"], check=True,
                   stdout=None if verbose else subprocess.DEVNULL)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ------------------------------------------------------------------------------------------
# ctypes mirrors of include/grtx.h
# ------------------------------------------------------------------------------------------
_fp = C.c_void_p


class grtx_gaussians(C.Structure):
    _fields_ = [("means", _fp), ("log_scales", _fp), ("quats", _fp), ("opacity_logits", _fp), ("sh", _fp),
                ("n", C.c_int64), ("sh_degree", C.c_int32), ("reserved", C.c_int32)]


class grtx_grads(C.Structure):
    _fields_ = [("means", _fp), ("log_scales", _fp), ("quats", _fp), ("opacity_logits", _fp), ("sh", _fp)]


class grtx_params(C.Structure):
    _fields_ = [("k", C.c_int32), ("traversal", C.c_int32), ("alpha_min", C.c_float), ("T_min", C.c_float),
                ("alpha_max", C.c_float), ("bg", C.c_float * 3), ("ckpt_capacity", C.c_int32),
                ("evict_capacity", C.c_int32), ("bvh_codes", C.c_int32), ("bvh_builder", C.c_int32),
                ("packet_stack", C.c_int32), ("bvh_width", C.c_int32), ("bvh_quantize", C.c_int32)]


class grtx_camera(C.Structure):
    _fields_ = [("type", C.c_int32), ("width", C.c_int32), ("height", C.c_int32), ("pos", C.c_float * 3),
                ("right", C.c_float * 3), ("up", C.c_float * 3), ("forward", C.c_float * 3), ("fov", C.c_float),
                ("t_near", C.c_float), ("t_far", C.c_float), ("ray_origins", _fp), ("ray_dirs", _fp),
                ("ray_tnear", _fp), ("ray_tfar", _fp)]


class grtx_stats(C.Structure):
    _fields_ = [(n, C.c_ulonglong) for n in ("rays", "nodes", "leaves", "blended", "rounds", "ckpt_writes",
                                             "evictions", "fallbacks", "stack_overflow", "collected",
                                             "bounds_errors")]


class grtx_saved(C.Structure):
    _fields_ = [("leaves", _fp), ("n", _fp), ("cap", C.c_int32), ("reserved", C.c_int32)]


class grtx_trace_outputs(C.Structure):
    _fields_ = [("rgbT", _fp), ("n_blended", _fp), ("blended_ids", _fp), ("ids_cap", C.c_int32),
                ("reserved", C.c_int32), ("stats", _fp), ("visits", _fp), ("visits_n", _fp),
                ("visits_cap", C.c_int32), ("visits_stride", C.c_int32), ("visits_rows", C.c_int32),
                ("reserved2", C.c_int32), ("saved", _fp)]


class grtx_scene_info(C.Structure):
    _fields_ = [("n_gaussians", C.c_int64), ("n_valid", C.c_int64), ("n_leaves", C.c_int64), ("n_nodes", C.c_int64),
                ("depth", C.c_int32), ("form", C.c_int32), ("sh_degree", C.c_int32), ("reserved", C.c_int32),
                ("bytes_nodes", C.c_int64), ("bytes_leaves", C.c_int64), ("bytes_appearance", C.c_int64),
                ("bytes_workspace", C.c_int64), ("bounds", C.c_float * 6)]


class grtx_mirror(C.Structure):
    _fields_ = [("center", C.c_float * 3), ("normal", C.c_float * 3), ("axis_u", C.c_float * 3),
                ("axis_v", C.c_float * 3), ("half_u", C.c_float), ("half_v", C.c_float),
                ("t_near_secondary", C.c_float), ("reserved", C.c_float)]


class grtx_glass(C.Structure):
    _fields_ = [("center", C.c_float * 3), ("radius", C.c_float), ("ior", C.c_float),
                ("t_near_secondary", C.c_float), ("reserved", C.c_float * 2)]


class grtx_instance(C.Structure):
    _fields_ = [("scene", _fp), ("object_to_world", C.c_float * 12), ("reserved", C.c_int32 * 2)]


class grtx_request(C.Structure):
    _fields_ = [("scene_id", C.c_int32), ("reserved", C.c_int32), ("cam", grtx_camera), ("d_rgbT", _fp),
                ("tag", C.c_uint64)]


class grtx_completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("reserved", C.c_int32), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("d_rgbT", _fp)]


class grtx_server_info(C.Structure):
    _fields_ = [("n_step_slots", C.c_int32), ("blocks_per_step", C.c_int32), ("list_bytes", C.c_int64),
                ("arena_bytes", C.c_int64), ("arena_used", C.c_int64), ("device_bytes", C.c_int64),
                ("n_inflight", C.c_int32), ("n_pending", C.c_int32), ("n_launches", C.c_int64),
                ("n_appends", C.c_int64), ("n_retried_tiles", C.c_int64)]


# every symbol declared in include/grtx.h with its ctypes signature
_SIGS = {
    "grtx_status_string": (C.c_char_p, [C.c_int]),
    "grtx_version": (C.c_int, []),
    "grtx_last_error": (C.c_char_p, []),
    "grtx_memory_trim": (C.c_int, [C.c_int64]),
    "grtx_prep_gaussians": (C.c_int, [C.POINTER(grtx_gaussians), C.c_float, _fp, _fp, _fp]),
    "grtx_morton_codes": (C.c_int, [_fp, C.c_int64, _fp, _fp, _fp, _fp]),
    "grtx_morton_codes_sized": (C.c_int, [_fp, C.c_int64, _fp, _fp, _fp, _fp]),
    "grtx_sort_pairs": (C.c_int, [_fp, _fp, C.c_int64, C.c_int, _fp, C.POINTER(C.c_size_t), _fp]),
    "grtx_radix_tree": (C.c_int, [_fp, C.c_int64, _fp, _fp, _fp, _fp]),
    "grtx_ploc_tree": (C.c_int, [_fp, C.c_int64, _fp, _fp, _fp, C.POINTER(C.c_int), _fp]),
    "grtx_refit": (C.c_int, [_fp, _fp, _fp, _fp, C.c_int64, _fp, _fp, _fp]),
    "grtx_build_bvh": (C.c_int, [C.POINTER(grtx_gaussians), C.POINTER(grtx_params), C.c_int, _fp, C.POINTER(_fp)]),
    "grtx_scene_update": (C.c_int, [_fp, C.POINTER(grtx_gaussians), C.c_int, _fp, C.POINTER(C.c_int)]),
    "grtx_scene_info_get": (C.c_int, [_fp, C.POINTER(grtx_scene_info)]),
    "grtx_scene_export": (C.c_int, [_fp, _fp, _fp, _fp, _fp]),
    "grtx_scene_destroy": (None, [_fp]),
    "grtx_generate_rays": (C.c_int, [C.POINTER(grtx_camera), _fp, _fp, _fp, _fp, _fp]),
    "grtx_trace_forward": (C.c_int, [_fp, C.POINTER(grtx_camera), C.POINTER(grtx_params),
                                     C.POINTER(grtx_trace_outputs), _fp]),
    "grtx_trace_forward_batch": (C.c_int, [_fp, C.POINTER(grtx_camera), C.c_int, C.POINTER(grtx_params),
                                           C.POINTER(_fp), _fp]),
    "grtx_trace_backward": (C.c_int, [_fp, C.POINTER(grtx_gaussians), C.POINTER(grtx_camera), C.POINTER(grtx_params),
                                      _fp, _fp, C.POINTER(grtx_grads), _fp]),
    "grtx_trace_backward_saved": (C.c_int, [_fp, C.POINTER(grtx_gaussians), C.POINTER(grtx_camera),
                                            C.POINTER(grtx_params), _fp, _fp, C.POINTER(grtx_saved),
                                            C.POINTER(grtx_grads), _fp]),
    "grtx_mirror_rays": (C.c_int, [C.POINTER(grtx_camera), C.POINTER(grtx_mirror)] + [_fp] * 11),
    "grtx_template_mesh": (C.c_int, [C.c_int, _fp, C.POINTER(C.c_int)]),
    "grtx_world_create": (C.c_int, [C.POINTER(grtx_instance), C.c_int, _fp, C.POINTER(_fp)]),
    "grtx_world_update": (C.c_int, [_fp, C.POINTER(grtx_instance), C.c_int, _fp]),
    "grtx_world_trace_forward": (C.c_int, [_fp, C.POINTER(grtx_camera), C.POINTER(grtx_params),
                                           C.POINTER(grtx_trace_outputs), _fp]),
    "grtx_world_destroy": (None, [_fp]),
    "grtx_secondary_rays": (C.c_int, [C.POINTER(grtx_camera), C.POINTER(grtx_mirror), C.c_int, C.POINTER(grtx_glass),
                                      C.c_int] + [_fp] * 11),
    "grtx_composite_bounce": (C.c_int, [_fp, _fp, _fp, _fp, C.c_int64, C.POINTER(C.c_float * 3), _fp]),
    "grtx_trace_forward_noalloc": (C.c_int, [_fp, C.POINTER(grtx_camera), C.POINTER(grtx_params), _fp, _fp]),
    "grtx_server_create": (C.c_int, [C.POINTER(_fp), C.c_int, C.POINTER(grtx_params), C.c_int64, C.c_int64, C.c_int,
                                     _fp, C.POINTER(_fp)]),
    "grtx_server_release": (C.c_int, [_fp, _fp]),
    "grtx_server_get_info": (C.c_int, [_fp, C.POINTER(grtx_server_info)]),
    "grtx_server_set_linger": (C.c_int, [_fp, C.c_int64]),
    "grtx_server_set_order": (C.c_int, [_fp, C.c_double]),
    "grtx_server_set_append_guard": (C.c_int, [_fp, C.c_int]),
    "grtx_server_submit": (C.c_int, [_fp, C.POINTER(grtx_request), C.c_int]),
    "grtx_server_poll": (C.c_int, [_fp, C.POINTER(grtx_completion), C.c_int, C.POINTER(C.c_int), C.c_int]),
    "grtx_render_requests": (C.c_int, [_fp, C.POINTER(grtx_request), C.c_int, C.POINTER(grtx_completion),
                                       C.POINTER(C.c_int), _fp]),
    "grtx_server_load": (C.c_int, [_fp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "grtx_server_destroy": (None, [_fp]),
}

SYMBOLS = tuple(_SIGS)


def lib():
    """The loaded library. Raises if it has not been built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(the CUDA extension is required; there is no CPU path)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _status_text(st: int) -> str:
    try:
        return lib().grtx_status_string(st).decode()
    except Exception:
        return "?"


def check(st: int, what: str):
    if st != 0:
        detail = lib().grtx_last_error().decode(errors="replace")
        raise GrtxError(st, what, detail)


# ------------------------------------------------------------------------------------------
# Argument helpers
# ------------------------------------------------------------------------------------------
def ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


class _DeviceArray:
    """A float32 device array the library owns, exposed through __cuda_array_interface__."""

    def __init__(self, address: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": "<f4",
                                         "data": (int(address), False), "version": 3, "strides": None}


def device_view(address: int, shape):
    """A torch tensor viewing float32 device memory owned by the library (no copy; valid as
    long as the library keeps the memory)."""
    import torch
    return torch.as_tensor(_DeviceArray(address, shape), device="cuda")


def stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


BVH_CODES = {"sized": 0, "centroid": 1}
BVH_BUILDERS = {"ploc": 0, "lbvh": 1}


def make_params(k=16, traversal=0, alpha_min=0.01, T_min=1e-3, alpha_max=0.99, bg=(0.0, 0.0, 0.0),
                ckpt_capacity=0, evict_capacity=0, bvh_codes=0, bvh_builder=0, packet_stack=0,
                bvh_width=0, bvh_quantize=0) -> grtx_params:
    p = grtx_params()
    p.packet_stack = int(packet_stack)
    p.bvh_width = int(bvh_width)
    p.bvh_quantize = int(bvh_quantize)
    p.bvh_codes = BVH_CODES[bvh_codes] if isinstance(bvh_codes, str) else int(bvh_codes)
    p.bvh_builder = BVH_BUILDERS[bvh_builder] if isinstance(bvh_builder, str) else int(bvh_builder)
    p.k, p.traversal = int(k), int(traversal)
    p.alpha_min, p.T_min, p.alpha_max = alpha_min, T_min, alpha_max
    for i in range(3):
        p.bg[i] = bg[i]
    p.ckpt_capacity, p.evict_capacity = int(ckpt_capacity), int(evict_capacity)
    return p


def make_camera(cam: dict, rays=None) -> grtx_camera:
    """A grtx_camera from a scenes.* camera dict, or (rays given) an explicit ray list:
    rays = (origins [n,3], dirs [n,3], t_near [n] or None, t_far [n] or None) CUDA tensors.
    With both, and the camera's width * height equal to n, the list is the camera's image of
    rays (row-major) and is traced in pixel tiles."""
    c = grtx_camera()
    if rays is not None:
        o, d, tn, tf = rays
        c.type = 2
        n = int(o.shape[0])
        if cam and "width" in cam and "height" in cam and int(cam["width"]) * int(cam["height"]) == n:
            c.width, c.height = int(cam["width"]), int(cam["height"])
        else:
            c.width, c.height = n, 1
        c.t_near = float(cam.get("t_near", 0.0)) if cam else 0.0
        c.t_far = float(cam.get("t_far", float("inf"))) if cam else float("inf")
        c.ray_origins, c.ray_dirs = ptr(o), ptr(d)
        c.ray_tnear, c.ray_tfar = ptr(tn), ptr(tf)
        return c
    c.type = int(cam["type"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    for name in ("pos", "right", "up", "forward"):
        arr = getattr(c, name)
        for i in range(3):
            arr[i] = float(cam[name][i])
    c.fov, c.t_near, c.t_far = float(cam["fov"]), float(cam["t_near"]), float(cam["t_far"])
    return c


def make_gaussians(means, log_scales, quats, logits, sh, sh_degree: int) -> grtx_gaussians:
    g = grtx_gaussians()
    for t in (means, log_scales, quats, logits, sh):
        assert t.is_cuda and t.is_contiguous() and t.dtype.is_floating_point and t.element_size() == 4
    g.means, g.log_scales, g.quats, g.opacity_logits, g.sh = (ptr(means), ptr(log_scales), ptr(quats), ptr(logits),
                                                             ptr(sh))
    g.n = int(logits.shape[0])
    g.sh_degree = int(sh_degree)
    return g


# ------------------------------------------------------------------------------------------
# Entry points with the ABI's names (tensors in, status checked)
# ------------------------------------------------------------------------------------------
def grtx_prep_gaussians(g: grtx_gaussians, alpha_min: float, geom, aabb, stream=None):
    check(lib().grtx_prep_gaussians(C.byref(g), alpha_min, ptr(geom), ptr(aabb), stream_handle(stream)),
          "grtx_prep_gaussians")


def grtx_morton_codes(aabb, bounds, codes, bounds_out=None, stream=None):
    check(lib().grtx_morton_codes(ptr(aabb), int(aabb.shape[0]), ptr(bounds), ptr(bounds_out), ptr(codes),
                                  stream_handle(stream)), "grtx_morton_codes")


def grtx_morton_codes_sized(aabb, bounds, codes, bounds_out=None, stream=None):
    check(lib().grtx_morton_codes_sized(ptr(aabb), int(aabb.shape[0]), ptr(bounds), ptr(bounds_out), ptr(codes),
                                        stream_handle(stream)), "grtx_morton_codes_sized")


def grtx_ploc_tree(leaf_aabb, left, right, parent, stream=None) -> int:
    it = C.c_int(0)
    check(lib().grtx_ploc_tree(ptr(leaf_aabb), int(leaf_aabb.shape[0]), ptr(left), ptr(right), ptr(parent),
                               C.byref(it), stream_handle(stream)), "grtx_ploc_tree")
    return it.value


def grtx_sort_pairs(keys, values, key_bits=64, stream=None):
    import torch
    n = int(keys.shape[0])
    nb = C.c_size_t(0)
    check(lib().grtx_sort_pairs(None, None, n, key_bits, None, C.byref(nb), None), "grtx_sort_pairs(size)")
    temp = torch.empty(int(nb.value), dtype=torch.uint8, device=keys.device)
    check(lib().grtx_sort_pairs(ptr(keys), ptr(values), n, key_bits, ptr(temp), C.byref(nb), stream_handle(stream)),
          "grtx_sort_pairs")
    return temp


def grtx_radix_tree(sorted_keys, left, right, parent, stream=None):
    check(lib().grtx_radix_tree(ptr(sorted_keys), int(sorted_keys.shape[0]), ptr(left), ptr(right), ptr(parent),
                                stream_handle(stream)), "grtx_radix_tree")


def grtx_refit(left, right, parent, leaf_aabb, node_aabb, counters, stream=None):
    check(lib().grtx_refit(ptr(left), ptr(right), ptr(parent), ptr(leaf_aabb), int(leaf_aabb.shape[0]),
                           ptr(node_aabb), ptr(counters), stream_handle(stream)), "grtx_refit")


def grtx_build_bvh(g: grtx_gaussians, p: grtx_params, form: int, stream=None) -> int:
    out = C.c_void_p()
    check(lib().grtx_build_bvh(C.byref(g), C.byref(p), int(form), stream_handle(stream), C.byref(out)),
          "grtx_build_bvh")
    return out.value


UPDATE_MODES = {"refit": 0, "rebuild": 1}


def grtx_scene_update(scene: int, g: grtx_gaussians, mode: int, stream=None) -> bool:
    """Update a scene in place for new parameters; True when it was rebuilt."""
    rebuilt = C.c_int(0)
    check(lib().grtx_scene_update(C.c_void_p(scene), C.byref(g), int(mode), stream_handle(stream), C.byref(rebuilt)),
          "grtx_scene_update")
    return bool(rebuilt.value)


def grtx_memory_trim(keep_bytes: int = 0):
    """Return the library pool's unused device memory beyond keep_bytes to the driver."""
    check(lib().grtx_memory_trim(int(keep_bytes)), "grtx_memory_trim")


def grtx_scene_info_get(scene: int) -> dict:
    info = grtx_scene_info()
    check(lib().grtx_scene_info_get(C.c_void_p(scene), C.byref(info)), "grtx_scene_info_get")
    d = {name: getattr(info, name) for name, _ in grtx_scene_info._fields_ if name not in ("reserved", "bounds")}
    d["bounds"] = list(info.bounds)
    return d


def grtx_scene_export(scene: int, nodes=None, leaf_ids=None, codes=None, stream=None):
    check(lib().grtx_scene_export(C.c_void_p(scene), ptr(nodes), ptr(leaf_ids), ptr(codes), stream_handle(stream)),
          "grtx_scene_export")


def grtx_scene_destroy(scene: int):
    if scene:
        lib().grtx_scene_destroy(C.c_void_p(scene))


def grtx_generate_rays(cam: grtx_camera, origins, dirs, tnear=None, tfar=None, stream=None):
    check(lib().grtx_generate_rays(C.byref(cam), ptr(origins), ptr(dirs), ptr(tnear), ptr(tfar),
                                   stream_handle(stream)), "grtx_generate_rays")


def make_saved(leaves, n) -> grtx_saved:
    """Saved blend lists: leaves [n_rays, cap] int32 and n [n_rays] int32 CUDA tensors."""
    sv = grtx_saved()
    sv.leaves, sv.n, sv.cap = ptr(leaves), ptr(n), int(leaves.shape[1])
    return sv


def grtx_trace_forward(scene: int, cam: grtx_camera, p: grtx_params, rgbT, n_blended=None, blended_ids=None,
                       stats=None, stream=None, visits=None, visits_n=None, visits_stride: int = 1, saved=None):
    """visits: optional [rows, cap] uint32/int32 device log of every visits_stride-th ray's node
    fetches, visits_n: [rows] their counts (see grtx_trace_outputs). saved: optional grtx_saved
    that receives the blend lists."""
    out = grtx_trace_outputs()
    if saved is not None:
        out.saved = C.addressof(saved)
    out.rgbT, out.n_blended, out.blended_ids = ptr(rgbT), ptr(n_blended), ptr(blended_ids)
    out.ids_cap = int(blended_ids.shape[-1]) if blended_ids is not None else 0
    out.stats = ptr(stats)
    if visits is not None:
        out.visits, out.visits_n = ptr(visits), ptr(visits_n)
        out.visits_rows, out.visits_cap = int(visits.shape[0]), int(visits.shape[1])
        out.visits_stride = int(visits_stride)
    check(lib().grtx_trace_forward(C.c_void_p(scene), C.byref(cam), C.byref(p), C.byref(out), stream_handle(stream)),
          "grtx_trace_forward")


def grtx_trace_forward_batch(scene: int, cams, p: grtx_params, outs, stream=None):
    """cams: list of grtx_camera; outs: matching list of rgbT tensors."""
    n = len(cams)
    arr = (grtx_camera * max(n, 1))(*cams)
    ptrs = (_fp * max(n, 1))(*[ptr(o) for o in outs])
    check(lib().grtx_trace_forward_batch(C.c_void_p(scene), arr, n, C.byref(p), ptrs, stream_handle(stream)),
          "grtx_trace_forward_batch")


def make_instances(placements) -> C.Array:
    """placements: iterable of (scene handle, 3x4 object-to-world matrix, row-major)."""
    import numpy as np
    pl = list(placements)
    arr = (grtx_instance * max(len(pl), 1))()
    for i, (h, M) in enumerate(pl):
        arr[i].scene = h
        m = np.asarray(M, dtype=np.float64).reshape(12)
        for k in range(12):
            arr[i].object_to_world[k] = float(m[k])
    return arr


def grtx_world_create(placements, stream=None) -> int:
    arr = make_instances(placements)
    out = C.c_void_p()
    check(lib().grtx_world_create(arr, len(list(placements)), stream_handle(stream), C.byref(out)),
          "grtx_world_create")
    return out.value


def grtx_world_update(world: int, placements, stream=None):
    arr = make_instances(placements)
    check(lib().grtx_world_update(C.c_void_p(world), arr, len(list(placements)), stream_handle(stream)),
          "grtx_world_update")


def grtx_world_trace_forward(world: int, cam: grtx_camera, p: grtx_params, rgbT, n_blended=None, blended_ids=None,
                             stats=None, stream=None):
    out = grtx_trace_outputs()
    out.rgbT, out.n_blended, out.blended_ids = ptr(rgbT), ptr(n_blended), ptr(blended_ids)
    out.ids_cap = int(blended_ids.shape[-1]) if blended_ids is not None else 0
    out.stats = ptr(stats)
    check(lib().grtx_world_trace_forward(C.c_void_p(world), C.byref(cam), C.byref(p), C.byref(out),
                                         stream_handle(stream)), "grtx_world_trace_forward")


def make_mirror(m: dict) -> grtx_mirror:
    g = grtx_mirror()
    for name in ("center", "normal", "axis_u", "axis_v"):
        arr = getattr(g, name)
        for i in range(3):
            arr[i] = float(m[name][i])
    g.half_u, g.half_v, g.t_near_secondary = float(m["half_u"]), float(m["half_v"]), float(m["t_near_secondary"])
    return g


def template_mesh(form: int):
    """Triangles [n][3][3] of the shared icosphere template of form 2 (ICO20) or 3 (ICO80)."""
    import numpy as np
    n = C.c_int(0)
    check(lib().grtx_template_mesh(int(form), None, C.byref(n)), "grtx_template_mesh")
    out = np.empty((n.value, 3, 3), dtype=np.float32)
    check(lib().grtx_template_mesh(int(form), out.ctypes.data, C.byref(n)), "grtx_template_mesh")
    return out


def make_glass(gl: dict) -> grtx_glass:
    g = grtx_glass()
    for i in range(3):
        g.center[i] = gl["center"][i]
    g.radius, g.ior, g.t_near_secondary = gl["radius"], gl["ior"], gl["t_near_secondary"]
    return g


def grtx_secondary_rays(cam: grtx_camera, mirrors, glass, prim, sec, sec_pixel, n_sec, stream=None):
    """mirrors / glass: lists of grtx_mirror / grtx_glass; prim, sec: (origins, dirs, tnear, tfar)."""
    ma = (grtx_mirror * max(len(mirrors), 1))(*mirrors)
    ga = (grtx_glass * max(len(glass), 1))(*glass)
    check(lib().grtx_secondary_rays(C.byref(cam), ma, len(mirrors), ga, len(glass), *[ptr(t) for t in prim],
                                    *[ptr(t) for t in sec], ptr(sec_pixel), ptr(n_sec), stream_handle(stream)),
          "grtx_secondary_rays")


def grtx_mirror_rays(cam: grtx_camera, mirror: grtx_mirror, prim, sec, sec_pixel, n_sec, stream=None):
    """prim / sec: (origins [n,3], dirs [n,3], tnear [n], tfar [n]) CUDA tensors."""
    check(lib().grtx_mirror_rays(C.byref(cam), C.byref(mirror), *[ptr(t) for t in prim], *[ptr(t) for t in sec],
                                 ptr(sec_pixel), ptr(n_sec), stream_handle(stream)), "grtx_mirror_rays")


def grtx_composite_bounce(rgbT, sec_rgbT, sec_pixel, n_sec, bg=(0.0, 0.0, 0.0), stream=None):
    b = (C.c_float * 3)(*bg)
    check(lib().grtx_composite_bounce(ptr(rgbT), ptr(sec_rgbT), ptr(sec_pixel), ptr(n_sec), int(sec_rgbT.shape[0]),
                                      C.byref(b), stream_handle(stream)), "grtx_composite_bounce")


def grtx_trace_forward_noalloc(scene: int, cam: grtx_camera, p: grtx_params, rgbT, stream=None):
    check(lib().grtx_trace_forward_noalloc(C.c_void_p(scene), C.byref(cam), C.byref(p), ptr(rgbT),
                                           stream_handle(stream)), "grtx_trace_forward_noalloc")


def grtx_trace_backward(scene: int, g: grtx_gaussians, cam: grtx_camera, p: grtx_params, rgbT, dL_drgbT,
                        grads: dict, stream=None):
    gr = grtx_grads()
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        setattr(gr, name, ptr(grads.get(name)))
    check(lib().grtx_trace_backward(C.c_void_p(scene), C.byref(g), C.byref(cam), C.byref(p), ptr(rgbT),
                                    ptr(dL_drgbT), C.byref(gr), stream_handle(stream)), "grtx_trace_backward")


def grtx_trace_backward_saved(scene: int, g: grtx_gaussians, cam: grtx_camera, p: grtx_params, rgbT, dL_drgbT,
                              saved: grtx_saved, grads: dict, stream=None):
    gr = grtx_grads()
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        setattr(gr, name, ptr(grads.get(name)))
    check(lib().grtx_trace_backward_saved(C.c_void_p(scene), C.byref(g), C.byref(cam), C.byref(p), ptr(rgbT),
                                          ptr(dL_drgbT), C.byref(saved), C.byref(gr), stream_handle(stream)),
          "grtx_trace_backward_saved")


STATS_FIELDS = tuple(n for n, _ in grtx_stats._fields_)


def stats_tensor(device="cuda"):
    import torch
    return torch.zeros(len(STATS_FIELDS), dtype=torch.int64, device=device)


def stats_dict(t) -> dict:
    v = t.cpu().tolist()
    return {n: int(v[i]) for i, n in enumerate(STATS_FIELDS)}
