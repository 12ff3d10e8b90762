"""User-facing API over libgrtx: scenes, rendering, and a torch.autograd.Function.

Tensors live on the current CUDA device; all work goes through the C ABI (native.py).
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as N

FORMS = {"sphere": 0, "proxy20": 1, "ico20": 2, "ico80": 3}
TRAVERSALS = {"checkpoint": 0, "restart": 1, "single": 2}


def _cuda_f32(a, device) -> torch.Tensor:
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return a.to(device=device, dtype=torch.float32).contiguous()


def params_to_device(g, device="cuda"):
    """(means, log_scales, quats, logits, sh) as contiguous float32 CUDA tensors."""
    return tuple(_cuda_f32(a, device) for a in (g.means, g.log_scales, g.quats, g.logits, g.sh))


class Scene:
    """A built acceleration structure (library-owned) for one set of Gaussians.

    form: "sphere" (one unit-sphere instance per Gaussian, Sec. IV-A), "ico20" / "ico80" (the
    same instances over a shared 20- / 80-triangle icosphere template, Sec. IV-A's second
    option) or "proxy20" (20 triangles per Gaussian in one monolithic BVH, the baseline of
    Sec. III-C)."""

    def __init__(self, means, log_scales, quats, logits, sh, sh_degree: int, form: str = "sphere",
                 alpha_min: float = 0.01, stream=None, bvh_codes: str = "sized", bvh_builder: str = "ploc",
                 bvh_width: int = 2, bvh_quantize: bool = False):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.tensors = tuple(_cuda_f32(a, dev) for a in (means, log_scales, quats, logits, sh))
        self.sh_degree = int(sh_degree)
        self.form = form
        self.alpha_min = float(alpha_min)
        self._g = N.make_gaussians(*self.tensors, self.sh_degree)
        self.bvh_codes = bvh_codes
        self.bvh_builder = bvh_builder
        self.bvh_width = int(bvh_width)
        p = N.make_params(alpha_min=alpha_min, bvh_codes=bvh_codes, bvh_builder=bvh_builder, bvh_width=bvh_width,
                          bvh_quantize=int(bool(bvh_quantize)))
        self.handle = N.grtx_build_bvh(self._g, p, FORMS[form], stream)

    @classmethod
    def from_params(cls, g, form="sphere", alpha_min=0.01, stream=None, bvh_codes="sized", bvh_builder="ploc",
                    bvh_width=2, bvh_quantize=False):
        return cls(g.means, g.log_scales, g.quats, g.logits, g.sh, g.sh_degree, form, alpha_min, stream, bvh_codes,
                   bvh_builder, bvh_width, bvh_quantize)

    def update(self, means, log_scales, quats, logits, sh, mode: str = "refit", stream=None) -> bool:
        """New parameters for the same Gaussians (same n and SH degree), in place: "refit" keeps
        the tree and refits its boxes (sphere and icosphere forms), "rebuild" builds it anew.
        A refit falls back to a rebuild when a Gaussian culled at the last build is now above
        alpha_min. Returns True when the tree was rebuilt. The image does not depend on which."""
        dev = self.tensors[0].device
        tensors = tuple(_cuda_f32(a, dev) for a in (means, log_scales, quats, logits, sh))
        g = N.make_gaussians(*tensors, self.sh_degree)
        rebuilt = N.grtx_scene_update(self.handle, g, N.UPDATE_MODES[mode], stream)
        self.tensors, self._g = tensors, g
        return rebuilt

    @property
    def n(self) -> int:
        return int(self.tensors[3].shape[0])

    def info(self) -> dict:
        return N.grtx_scene_info_get(self.handle)

    def export(self):
        info = self.info()
        dev = self.tensors[0].device
        nodes = torch.empty((max(info["n_nodes"], 1), 16), dtype=torch.float32, device=dev)
        ids = torch.empty(max(info["n_leaves"], 1), dtype=torch.int32, device=dev)
        codes = torch.empty(max(info["n_leaves"], 1), dtype=torch.int64, device=dev)
        N.grtx_scene_export(self.handle, nodes, ids, codes)
        return nodes[: info["n_nodes"]], ids[: info["n_leaves"]], codes[: info["n_leaves"]]

    def close(self):
        if getattr(self, "handle", None):
            N.grtx_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class World:
    """Placed objects (Sec. VI multi-level instancing): each placement is (Scene, 3x4
    object-to-world matrix). The scenes are not owned and must outlive the world."""

    def __init__(self, placements, stream=None):
        self.placements = [(sc, np.asarray(M, dtype=np.float64).reshape(3, 4)) for sc, M in placements]
        self.alpha_min = self.placements[0][0].alpha_min
        self.handle = N.grtx_world_create([(sc.handle, M) for sc, M in self.placements], stream)

    def update(self, placements, stream=None):
        self.placements = [(sc, np.asarray(M, dtype=np.float64).reshape(3, 4)) for sc, M in placements]
        N.grtx_world_update(self.handle, [(sc.handle, M) for sc, M in self.placements], stream)

    def close(self):
        if getattr(self, "handle", None):
            N.lib().grtx_world_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render_world(world: World, cam: dict | None, rays=None, out=None, ids_cap: int = 0, want_n_blended=False,
                 want_stats=False, stream=None, **params):
    """Forward trace through a world. Returns dict(rgbT, n_blended?, ids? (world ids), stats?)."""
    p = trace_params(alpha_min=world.alpha_min, **params)
    c = N.make_camera(cam, rays)
    n = n_rays_of(cam, rays)
    dev = torch.device("cuda", torch.cuda.current_device())
    rgbT = out if out is not None else torch.empty((n, 4), dtype=torch.float32, device=dev)
    nb = torch.empty(n, dtype=torch.int32, device=dev) if want_n_blended else None
    ids = torch.empty((n, ids_cap), dtype=torch.int32, device=dev) if ids_cap > 0 else None
    st = N.stats_tensor(dev) if want_stats else None
    N.grtx_world_trace_forward(world.handle, c, p, rgbT, nb, ids, st, stream)
    res = {"rgbT": rgbT}
    if nb is not None:
        res["n_blended"] = nb
    if ids is not None:
        res["ids"] = ids
    if st is not None:
        res["stats"] = st
    return res


def trace_params(k=16, traversal="checkpoint", alpha_min=0.01, T_min=1e-3, alpha_max=0.99, bg=(0.0, 0.0, 0.0),
                 ckpt_capacity=0, evict_capacity=0, packet_stack=0, bvh_width=0):
    return N.make_params(k, TRAVERSALS[traversal] if isinstance(traversal, str) else traversal, alpha_min, T_min,
                         alpha_max, bg, ckpt_capacity, evict_capacity, packet_stack=packet_stack, bvh_width=bvh_width)


def n_rays_of(cam: dict, rays=None) -> int:
    return int(rays[0].shape[0]) if rays is not None else int(cam["width"]) * int(cam["height"])


def render(scene: Scene, cam: dict | None, rays=None, out=None, ids_cap: int = 0, want_n_blended=False,
           want_stats=False, stream=None, visit_log=None, save_cap: int = 0, **params):
    """Forward trace. Returns dict(rgbT [n_rays, 4], n_blended?, ids?, stats?, visits?,
    visits_n?, saved?). visit_log = (stride, rows, cap) logs the node fetches of every
    stride-th ray (output index), up to rows rays and cap fetches each. save_cap > 0 saves each
    ray's blend list (up to save_cap entries) for backward(saved=...)."""
    p = trace_params(alpha_min=scene.alpha_min, **params)
    c = N.make_camera(cam, rays)
    n = n_rays_of(cam, rays)
    dev = scene.tensors[0].device
    rgbT = out if out is not None else torch.empty((n, 4), dtype=torch.float32, device=dev)
    nb = torch.empty(n, dtype=torch.int32, device=dev) if want_n_blended else None
    ids = torch.empty((n, ids_cap), dtype=torch.int32, device=dev) if ids_cap > 0 else None
    st = N.stats_tensor(dev) if want_stats else None
    vis = vis_n = None
    stride = 1
    if visit_log is not None:
        stride, rows, cap = (int(v) for v in visit_log)
        vis = torch.empty((rows, cap), dtype=torch.int32, device=dev)
        vis_n = torch.empty(rows, dtype=torch.int32, device=dev)
    saved = sv = None
    if save_cap > 0:
        saved = (torch.empty((n, int(save_cap)), dtype=torch.int32, device=dev),
                 torch.empty(n, dtype=torch.int32, device=dev))
        sv = N.make_saved(*saved)
    N.grtx_trace_forward(scene.handle, c, p, rgbT, nb, ids, st, stream, vis, vis_n, stride, saved=sv)
    res = {"rgbT": rgbT}
    if saved is not None:
        res["saved"] = saved
    if nb is not None:
        res["n_blended"] = nb
    if ids is not None:
        res["ids"] = ids
    if st is not None:
        res["stats"] = st
    if vis is not None:
        res["visits"], res["visits_n"] = vis, vis_n
    return res


def render_batch(scene: Scene, views, stream=None, **params) -> list:
    """Several views of one scene in one launch: views = [(cam, rays)] with cam a camera dict
    or None and rays an explicit ray list or None (as in render). Returns the rgbT of each."""
    p = trace_params(alpha_min=scene.alpha_min, **params)
    dev = scene.tensors[0].device
    cams, outs = [], []
    for cam, rays in views:
        cams.append(N.make_camera(cam, rays))
        outs.append(torch.empty((n_rays_of(cam, rays), 4), dtype=torch.float32, device=dev))
    N.grtx_trace_forward_batch(scene.handle, cams, p, outs, stream)
    return outs


def visit_counts(visits, visits_n) -> dict:
    """Per logged ray: node and leaf fetches, total and distinct, from a visit log
    (numpy or torch; rows whose count exceeds the log's width are left out)."""
    import numpy as np
    V = visits.cpu().numpy() if hasattr(visits, "cpu") else np.asarray(visits)
    n = visits_n.cpu().numpy() if hasattr(visits_n, "cpu") else np.asarray(visits_n)
    V = V.view(np.uint32)
    rows = [r for r in range(V.shape[0]) if 0 < n[r] <= V.shape[1]]
    tot = np.array([n[r] for r in rows], dtype=np.int64)
    uniq = np.array([len(np.unique(V[r, : n[r]])) for r in rows], dtype=np.int64)
    return {"rays": len(rows), "truncated": int((n > V.shape[1]).sum()), "fetches_per_ray": float(tot.mean()) if rows else 0.0,
            "distinct_per_ray": float(uniq.mean()) if rows else 0.0,
            "revisit_fraction": float(1.0 - uniq.sum() / tot.sum()) if rows and tot.sum() else 0.0}


def backward(scene: Scene, cam: dict | None, rgbT, dL_drgbT, rays=None, stream=None, saved=None, **params):
    """Gradients of the raw parameters the scene was built from, given dL/d(rgbT). saved: the
    blend lists of render(save_cap=...) for this view: rays with a complete list skip the
    traversal."""
    p = trace_params(alpha_min=scene.alpha_min, **params)
    c = N.make_camera(cam, rays)
    grads = {name: torch.zeros_like(t) for name, t in
             zip(("means", "log_scales", "quats", "opacity_logits", "sh"), scene.tensors)}
    if saved is None:
        N.grtx_trace_backward(scene.handle, scene._g, c, p, rgbT.contiguous(), dL_drgbT.contiguous(), grads, stream)
    else:
        N.grtx_trace_backward_saved(scene.handle, scene._g, c, p, rgbT.contiguous(), dL_drgbT.contiguous(),
                                    N.make_saved(*saved), grads, stream)
    return grads


class RenderFunction(torch.autograd.Function):
    """Differentiable render: brings the BVH up to the current parameters, traces forward,
    and in backward re-traverses the same rounds to accumulate parameter gradients. Without a
    scene in opts the BVH is built anew at every call (the faster-to-build radix tree "lbvh"
    by default; opts may set bvh_builder / bvh_codes) and freed after backward. With
    opts["scene"] (a sphere- or icosphere-form Scene of the same Gaussians, kept by the caller
    across steps) it is updated in place, by opts["update"] = "refit" (default) or
    "rebuild". With opts["save_cap"] > 0 the forward saves each ray's blend list (up to that
    many entries) and the backward reads it instead of re-traversing, replaying only the rays
    whose list overflowed."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, logits, sh, sh_degree, cam, opts):
        o = dict(opts)
        params = (means.detach(), log_scales.detach(), quats.detach(), logits.detach(), sh.detach())
        scene = o.pop("scene", None)
        mode = o.pop("update", "refit")
        ctx.owned = scene is None
        if scene is None:
            scene = Scene(*params, sh_degree, "sphere", o.pop("alpha_min", 0.01), bvh_codes=o.pop("bvh_codes", "sized"),
                          bvh_builder=o.pop("bvh_builder", "lbvh"))
        else:
            if scene.sh_degree != int(sh_degree):
                raise ValueError("the scene's SH degree differs from sh_degree")
            for key in ("alpha_min", "bvh_codes", "bvh_builder"):
                o.pop(key, None)
            scene.update(*params, mode=mode)
        save_cap = int(o.pop("save_cap", 0))
        res = render(scene, cam, save_cap=save_cap, **o)
        rgbT = res["rgbT"]
        ctx.scene, ctx.cam, ctx.opts, ctx.saved = scene, cam, o, res.get("saved")
        ctx.save_for_backward(rgbT)
        return rgbT

    @staticmethod
    def backward(ctx, grad_rgbT):
        (rgbT,) = ctx.saved_tensors
        g = backward(ctx.scene, ctx.cam, rgbT, grad_rgbT.float().contiguous(), saved=ctx.saved, **ctx.opts)
        ctx.saved = None
        if ctx.owned:
            ctx.scene.close()
        return g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"], None, None, None


def render_differentiable(means, log_scales, quats, logits, sh, sh_degree: int, cam: dict, **opts):
    return RenderFunction.apply(means, log_scales, quats, logits, sh, sh_degree, cam, opts)
