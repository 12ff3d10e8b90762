"""ctypes wrapper of the FP64 CPU oracle in ``grtx_oracle.c``.

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may use it; the library's product path never does. It shares no code with
the CUDA implementation. Every entry point takes and returns NumPy float64 arrays (the
Morton/radix/refit helpers use float32 / uint64 / uint32, matching their definitions).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grtx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgrtx_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class OgCamera(C.Structure):
    _fields_ = [("type", C.c_int), ("width", C.c_int), ("height", C.c_int),
                ("pos", C.c_double * 3), ("right", C.c_double * 3), ("up", C.c_double * 3),
                ("forward", C.c_double * 3), ("fov", C.c_double), ("t_near", C.c_double),
                ("t_far", C.c_double)]


class OgParams(C.Structure):
    _fields_ = [("alpha_min", C.c_double), ("T_min", C.c_double), ("alpha_max", C.c_double),
                ("bg", C.c_double * 3)]


class OgRoundCfg(C.Structure):
    _fields_ = [("k", C.c_int), ("checkpoint", C.c_int), ("ckpt_cap", C.c_int),
                ("evict_cap", C.c_int)]


class OgRoundStats(C.Structure):
    _fields_ = [(n, C.c_longlong) for n in
                ("nodes", "leaves", "rounds", "ckpt_writes", "evictions", "fallbacks", "unique_nodes")]


class OgMirror(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("normal", C.c_double * 3), ("axis_u", C.c_double * 3),
                ("axis_v", C.c_double * 3), ("half_u", C.c_double), ("half_v", C.c_double),
                ("t_near_secondary", C.c_double)]


class OgGlass(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("radius", C.c_double), ("ior", C.c_double),
                ("t_near_secondary", C.c_double)]


class OgGrads(C.Structure):
    _fields_ = [(n, C.POINTER(C.c_double)) for n in ("means", "log_scales", "quats", "logits", "sh")]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_fp = C.POINTER(C.c_float)
_u64p = C.POINTER(C.c_uint64)
_u32p = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.og_scene_create.restype = C.c_void_p
            L.og_scene_create.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_double]
            L.og_scene_free.argtypes = [C.c_void_p]
            L.og_scene_export.argtypes = [C.c_void_p] + [_dp] * 7 + [_ip]
            L.og_unit_sphere_test.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp]
            L.og_response_one.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp]
            L.og_sh_basis.argtypes = [C.c_int, _dp, _dp]
            L.og_camera_rays.argtypes = [C.POINTER(OgCamera), _dp, _dp, _dp, _dp]
            L.og_render.argtypes = [C.c_void_p, C.POINTER(OgParams), C.c_int, _dp, _dp, _dp, _dp, _dp,
                                    _ip, _ip, C.c_int, _ip]
            L.og_num_threads.restype = C.c_int
            L.og_kbuf_insert.restype = C.c_int
            L.og_kbuf_insert.argtypes = [_dp, _ip, _ip, C.c_int, C.c_double, C.c_int, _dp, _ip]
            L.og_bvh_build.restype = C.c_void_p
            L.og_bvh_build.argtypes = [C.c_void_p]
            L.og_bvh_free.argtypes = [C.c_void_p]
            L.og_bvh_num_nodes.restype = C.c_int
            L.og_bvh_num_nodes.argtypes = [C.c_void_p]
            L.og_render_rounds.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(OgParams),
                                           C.POINTER(OgRoundCfg), C.c_int, _dp, _dp, _dp, _dp, _dp,
                                           _ip, C.POINTER(OgRoundStats), C.c_int]
            L.og_backward.argtypes = [C.c_void_p, C.POINTER(OgParams), C.c_int, _dp, _dp, _dp, _dp, _dp,
                                      C.POINTER(OgGrads), C.POINTER(OgGrads)]
            L.og_mirror_rays.restype = C.c_int
            L.og_mirror_rays.argtypes = [C.POINTER(OgCamera), C.POINTER(OgMirror)] + [_dp] * 8 + [_ip]
            L.og_composite_bounce.argtypes = [_dp, _dp, _ip, C.c_int, _dp]
            L.og_world_render.argtypes = [C.POINTER(C.c_void_p), C.c_int, _ip, _dp, C.POINTER(OgParams), C.c_int,
                                          _dp, _dp, _dp, _dp, _dp, _ip, _ip, C.c_int, _ip]
            L.og_secondary_rays.restype = C.c_int
            L.og_secondary_rays.argtypes = ([C.POINTER(OgCamera), C.POINTER(OgMirror), C.c_int, C.POINTER(OgGlass),
                                             C.c_int] + [_dp] * 8 + [_ip])
            L.og_centroid_bounds.argtypes = [C.c_int, _fp, _fp]
            L.og_morton63.argtypes = [C.c_int, _fp, _fp, _u64p]
            L.og_morton_sized64.argtypes = [C.c_int, _fp, _fp, _u64p]
            L.og_radix_tree.argtypes = [C.c_int, _u64p, _u32p, _u32p]
            L.og_refit.argtypes = [C.c_int, _u32p, _u32p, _fp, _fp]
            L.og_ploc.restype = C.c_int
            L.og_ploc.argtypes = [C.c_int, _fp, C.c_int, _u32p, _u32p]
            _lib = L
    return _lib


def _p(a: np.ndarray, ty=_dp):
    return a.ctypes.data_as(ty)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(lib().og_num_threads())


def make_params(alpha_min=0.01, T_min=1e-3, alpha_max=0.99, bg=(0.0, 0.0, 0.0)) -> OgParams:
    p = OgParams()
    p.alpha_min, p.T_min, p.alpha_max = alpha_min, T_min, alpha_max
    for i in range(3):
        p.bg[i] = bg[i]
    return p


def make_camera(cam: dict) -> OgCamera:
    c = OgCamera()
    c.type = int(cam["type"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    for name in ("pos", "right", "up", "forward"):
        arr = getattr(c, name)
        for i in range(3):
            arr[i] = float(cam[name][i])
    c.fov, c.t_near, c.t_far = float(cam["fov"]), float(cam["t_near"]), float(cam["t_far"])
    return c


def camera_rays(cam: dict):
    """(origins, dirs, t_near, t_far) of every pixel, row-major from the top-left pixel."""
    c = make_camera(cam)
    n = c.width * c.height
    o = np.empty((n, 3)); d = np.empty((n, 3)); tn = np.empty(n); tf = np.empty(n)
    lib().og_camera_rays(C.byref(c), _p(o), _p(d), _p(tn), _p(tf))
    return o, d, tn, tf


def sh_basis(degree: int, direction) -> np.ndarray:
    d = _f64(direction)
    Y = np.zeros(16)
    lib().og_sh_basis(int(degree), _p(d), _p(Y))
    return Y[: (degree + 1) ** 2]


def kbuf_insert(kt: np.ndarray, kid: np.ndarray, cnt: int, k: int, t: float, i: int):
    """In-place insertion into a k-buffer; returns (new count, rejected or None)."""
    c = C.c_int(cnt)
    rt = C.c_double(0.0)
    ri = C.c_int(0)
    rej = lib().og_kbuf_insert(_p(kt), _p(kid, _ip), C.byref(c), int(k), float(t), int(i),
                               C.byref(rt), C.byref(ri))
    return c.value, ((rt.value, ri.value) if rej else None)


class Scene:
    """FP64 oracle scene built from raw Gaussian parameters (float arrays of any dtype)."""

    def __init__(self, means, log_scales, quats, logits, sh, sh_degree: int, alpha_min=0.01):
        self.n = int(np.asarray(logits).shape[0])
        self.sh_degree = int(sh_degree)
        self.n_coef = (self.sh_degree + 1) ** 2
        self._keep = [_f64(means).reshape(-1, 3), _f64(log_scales).reshape(-1, 3),
                      _f64(quats).reshape(-1, 4), _f64(logits).reshape(-1),
                      _f64(sh).reshape(self.n, self.n_coef, 3)]
        m, ls, q, lg, s = self._keep
        self._h = lib().og_scene_create(self.n, self.sh_degree, _p(m), _p(ls), _p(q), _p(lg), _p(s),
                                        float(alpha_min))
        if not self._h:
            raise MemoryError("oracle scene allocation failed")
        self._bvh = None

    @classmethod
    def from_params(cls, g, alpha_min=0.01):
        return cls(g.means, g.log_scales, g.quats, g.logits, g.sh, g.sh_degree, alpha_min)

    def __del__(self):
        L = _lib
        if L is not None:
            if getattr(self, "_bvh", None):
                L.og_bvh_free(self._bvh)
            if getattr(self, "_h", None):
                L.og_scene_free(self._h)

    def export(self) -> dict:
        n = self.n
        out = dict(o=np.empty(n), s=np.empty((n, 3)), R=np.empty((n, 3, 3)), P=np.empty((n, 3, 3)),
                   kappa=np.empty(n), A=np.empty((n, 3, 4)), aabb=np.empty((n, 6)),
                   valid=np.empty(n, dtype=np.int32))
        lib().og_scene_export(self._h, *[_p(out[k]) for k in ("o", "s", "R", "P", "kappa", "A", "aabb")],
                              _p(out["valid"], _ip))
        out["valid"] = out["valid"].astype(bool)
        return out

    def response(self, i: int, ro, rd):
        """(t_alpha, d2, alpha) of Gaussian i for one ray (Eq. t-max-resp)."""
        r = np.empty(3)
        lib().og_response_one(self._h, int(i), _p(_f64(ro)), _p(_f64(rd)), _p(r))
        return float(r[0]), float(r[1]), float(r[2])

    def unit_sphere(self, i: int, ro, rd):
        """(t_alpha, D2) of Gaussian i through the unit-sphere transform."""
        t = C.c_double(); D2 = C.c_double()
        lib().og_unit_sphere_test(self._h, int(i), _p(_f64(ro)), _p(_f64(rd)), C.byref(t), C.byref(D2))
        return t.value, D2.value

    def render(self, rays, params: OgParams | None = None, ids_cap: int = 0):
        o, d, tn, tf = [_f64(a) for a in rays]
        n = tn.shape[0]
        params = params or make_params()
        out = np.empty((n, 4)); nb = np.empty(n, dtype=np.int32); nh = np.empty(n, dtype=np.int32)
        ids = np.full((n, max(ids_cap, 1)), -1, dtype=np.int32)
        lib().og_render(self._h, C.byref(params), n, _p(o), _p(d), _p(tn), _p(tf), _p(out),
                        _p(nb, _ip), _p(ids, _ip) if ids_cap > 0 else None, int(ids_cap), _p(nh, _ip))
        res = dict(out=out, n_blend=nb, n_hits=nh)
        if ids_cap > 0:
            res["ids"] = ids
        return res

    def bvh(self):
        if self._bvh is None:
            self._bvh = lib().og_bvh_build(self._h)
        return self._bvh

    def render_rounds(self, rays, params: OgParams | None = None, k: int = 8, checkpoint: bool = True,
                      ckpt_cap: int = -1, evict_cap: int = -1, count_unique: bool = False):
        o, d, tn, tf = [_f64(a) for a in rays]
        n = tn.shape[0]
        params = params or make_params()
        cfg = OgRoundCfg(int(k), int(bool(checkpoint)), int(ckpt_cap), int(evict_cap))
        out = np.empty((n, 4)); nb = np.empty(n, dtype=np.int32)
        st = OgRoundStats()
        lib().og_render_rounds(self._h, self.bvh(), C.byref(params), C.byref(cfg), n, _p(o), _p(d),
                               _p(tn), _p(tf), _p(out), _p(nb, _ip), C.byref(st), int(bool(count_unique)))
        stats = {name: int(getattr(st, name)) for name, _ in OgRoundStats._fields_}
        return dict(out=out, n_blend=nb, stats=stats)

    def backward(self, rays, dL_drgbT, params: OgParams | None = None, term_scale: bool = False) -> dict:
        """Analytic gradient of sum(dL_drgbT * image) w.r.t. the raw parameters. With
        term_scale, the result also holds "<name>_scale": per element, the summed magnitudes
        of the terms the element is formed from (see og_backward), the scale of its rounding
        error in a lower-precision evaluation."""
        o, d, tn, tf = [_f64(a) for a in rays]
        n = tn.shape[0]
        params = params or make_params()
        gL = _f64(dL_drgbT).reshape(n, 4)
        names = ("means", "log_scales", "quats", "logits", "sh")

        def zeros():
            return dict(means=np.zeros((self.n, 3)), log_scales=np.zeros((self.n, 3)), quats=np.zeros((self.n, 4)),
                        logits=np.zeros(self.n), sh=np.zeros((self.n, self.n_coef, 3)))
        g = zeros()
        G = OgGrads(*[_p(g[k]) for k in names])
        ga = zeros() if term_scale else None
        GA = OgGrads(*[_p(ga[k]) for k in names]) if term_scale else None
        lib().og_backward(self._h, C.byref(params), n, _p(o), _p(d), _p(tn), _p(tf), _p(gL), C.byref(G),
                          C.byref(GA) if term_scale else None)
        if term_scale:
            g.update({k + "_scale": ga[k] for k in names})
        return g


def world_render(scenes, inst_scene, object_to_world, rays, params: OgParams | None = None, ids_cap: int = 0):
    """Render rays through a world: instance i places scenes[inst_scene[i]] with the 3x4
    object-to-world map object_to_world[i] (row-major); ids are world ids."""
    o, d, tn, tf = [_f64(a) for a in rays]
    n = tn.shape[0]
    params = params or make_params()
    M = np.ascontiguousarray(np.asarray(object_to_world, dtype=np.float64).reshape(-1, 12))
    inst = np.ascontiguousarray(np.asarray(inst_scene, dtype=np.int32))
    handles = (C.c_void_p * max(len(scenes), 1))(*[s._h for s in scenes])
    out = np.empty((n, 4)); nb = np.empty(n, dtype=np.int32); nh = np.empty(n, dtype=np.int32)
    ids = np.full((n, max(ids_cap, 1)), -1, dtype=np.int32)
    lib().og_world_render(handles, len(inst), _p(inst, _ip), _p(M), C.byref(params), n, _p(o), _p(d), _p(tn),
                          _p(tf), _p(out), _p(nb, _ip), _p(ids, _ip) if ids_cap > 0 else None, int(ids_cap),
                          _p(nh, _ip))
    res = dict(out=out, n_blend=nb, n_hits=nh)
    if ids_cap > 0:
        res["ids"] = ids
    return res


def centroid_bounds(aabb_f32: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(aabb_f32, dtype=np.float32).reshape(-1, 6)
    b = np.empty(6, dtype=np.float32)
    lib().og_centroid_bounds(a.shape[0], _p(a, _fp), _p(b, _fp))
    return b


def morton63(aabb_f32: np.ndarray, bounds_f32: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(aabb_f32, dtype=np.float32).reshape(-1, 6)
    b = np.ascontiguousarray(bounds_f32, dtype=np.float32).reshape(6)
    codes = np.empty(a.shape[0], dtype=np.uint64)
    lib().og_morton63(a.shape[0], _p(a, _fp), _p(b, _fp), _p(codes, _u64p))
    return codes


def morton_sized64(aabb_f32: np.ndarray, bounds_f32: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(aabb_f32, dtype=np.float32).reshape(-1, 6)
    b = np.ascontiguousarray(bounds_f32, dtype=np.float32).reshape(6)
    codes = np.empty(a.shape[0], dtype=np.uint64)
    lib().og_morton_sized64(a.shape[0], _p(a, _fp), _p(b, _fp), _p(codes, _u64p))
    return codes


LEAF = 0x80000000


def radix_tree(sorted_codes: np.ndarray):
    k = np.ascontiguousarray(sorted_codes, dtype=np.uint64)
    n = k.shape[0]
    left = np.zeros(max(n - 1, 0), dtype=np.uint32)
    right = np.zeros(max(n - 1, 0), dtype=np.uint32)
    if n >= 2:
        lib().og_radix_tree(n, _p(k, _u64p), _p(left, _u32p), _p(right, _u32p))
    return left, right


def ploc(leaf_aabb_f32: np.ndarray, radius: int = 16):
    """(left, right, iterations) of the locally-ordered clustering tree over boxes in order."""
    a = np.ascontiguousarray(leaf_aabb_f32, dtype=np.float32).reshape(-1, 6)
    n = a.shape[0]
    left = np.zeros(max(n - 1, 0), dtype=np.uint32)
    right = np.zeros(max(n - 1, 0), dtype=np.uint32)
    it = lib().og_ploc(n, _p(a, _fp), int(radius), _p(left, _u32p), _p(right, _u32p)) if n >= 2 else 0
    return left, right, it


def refit(left: np.ndarray, right: np.ndarray, leaf_aabb_f32: np.ndarray) -> np.ndarray:
    la = np.ascontiguousarray(leaf_aabb_f32, dtype=np.float32).reshape(-1, 6)
    n = la.shape[0]
    node = np.zeros((max(n - 1, 0), 6), dtype=np.float32)
    if n >= 2:
        lib().og_refit(n, _p(np.ascontiguousarray(left, dtype=np.uint32), _u32p),
                       _p(np.ascontiguousarray(right, dtype=np.uint32), _u32p), _p(la, _fp), _p(node, _fp))
    return node


def make_mirror(m: dict) -> OgMirror:
    g = OgMirror()
    for name in ("center", "normal", "axis_u", "axis_v"):
        arr = getattr(g, name)
        for i in range(3):
            arr[i] = float(m[name][i])
    g.half_u, g.half_v, g.t_near_secondary = float(m["half_u"]), float(m["half_v"]), float(m["t_near_secondary"])
    return g


def mirror_rays(cam: dict, mirror: dict):
    """(primary rays, secondary rays, secondary pixel indices): primaries clipped at the mirror."""
    c = make_camera(cam)
    n = c.width * c.height
    prim = [np.empty((n, 3)), np.empty((n, 3)), np.empty(n), np.empty(n)]
    sec = [np.empty((n, 3)), np.empty((n, 3)), np.empty(n), np.empty(n)]
    spix = np.empty(n, dtype=np.int32)
    ns = lib().og_mirror_rays(C.byref(c), C.byref(make_mirror(mirror)), *[_p(a) for a in prim],
                              *[_p(a) for a in sec], _p(spix, _ip))
    return tuple(prim), tuple(a[:ns] for a in sec), spix[:ns].copy()


def make_glass(gl: dict) -> OgGlass:
    g = OgGlass()
    for i in range(3):
        g.center[i] = gl["center"][i]
    g.radius, g.ior, g.t_near_secondary = gl["radius"], gl["ior"], gl["t_near_secondary"]
    return g


def secondary_rays(cam: dict, mirrors=(), glass=()):
    """Primary rays clipped at the nearest mirror or glass ball, and one reflected or refracted
    secondary ray per such primary (pixel order); returns (prim, sec, spix)."""
    n = cam["width"] * cam["height"]
    po, pd = np.empty((n, 3)), np.empty((n, 3))
    ptn, ptf = np.empty(n), np.empty(n)
    so, sd = np.empty((n, 3)), np.empty((n, 3))
    stn, stf = np.empty(n), np.empty(n)
    spix = np.empty(n, dtype=np.int32)
    ma = (OgMirror * max(len(mirrors), 1))(*[make_mirror(m) for m in mirrors])
    ga = (OgGlass * max(len(glass), 1))(*[make_glass(g) for g in glass])
    c = make_camera(cam)
    ns = lib().og_secondary_rays(C.byref(c), ma, len(mirrors), ga, len(glass), _p(po), _p(pd), _p(ptn), _p(ptf),
                                 _p(so), _p(sd), _p(stn), _p(stf), _p(spix, _ip))
    return (po, pd, ptn, ptf), (so[:ns], sd[:ns], stn[:ns], stf[:ns]), spix[:ns]


def composite_bounce(rgbT: np.ndarray, sec_rgbT: np.ndarray, spix: np.ndarray, bg=(0.0, 0.0, 0.0)) -> np.ndarray:
    out = np.ascontiguousarray(rgbT, dtype=np.float64).copy()
    sec = np.ascontiguousarray(sec_rgbT, dtype=np.float64)
    sp = np.ascontiguousarray(spix, dtype=np.int32)
    b = np.asarray(bg, dtype=np.float64)
    lib().og_composite_bounce(_p(out), _p(sec), _p(sp, _ip), int(sp.shape[0]), _p(b))
    return out
