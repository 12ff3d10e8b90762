"""Seeded synthetic scenes, cameras and request streams.

This module only draws inputs: raw Gaussian parameters (means, log-scales, quaternions,
opacity logits, SH coefficients), camera descriptions and request arrival times. It holds
none of the rendering arithmetic, so both the CUDA path and the CPU oracle take their
inputs from here. The paper's trained scenes (Tanks&Temples, Mip-NeRF 360, Deep Blending;
0.76-2.43M Gaussians, Sec. V-A, Table "Summary of workloads") are not available, so these
generators stand in for them with the same scale of Gaussian counts and resolutions.

All arrays are float32, C-contiguous, structure of arrays:
  means (N,3), log_scales (N,3), quats (N,4) as (w,x,y,z), logits (N,), sh (N,(L+1)^2,3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_SQRT_PI = 2.0 * math.sqrt(math.pi)   # 1 / Y_00: the degree-0 coefficient of colour c is (c-0.5)*this


@dataclass
class GaussianParams:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.logits.shape[0])

    def arrays(self):
        return self.means, self.log_scales, self.quats, self.logits, self.sh

    def subset(self, idx) -> "GaussianParams":
        idx = np.asarray(idx)
        return GaussianParams(*(np.ascontiguousarray(a[idx]) for a in self.arrays()), self.sh_degree,
                              dict(self.meta))

    def copy(self) -> "GaussianParams":
        return GaussianParams(*(a.copy() for a in self.arrays()), self.sh_degree, dict(self.meta))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _normalize(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _logit(o: np.ndarray) -> np.ndarray:
    return np.log(o) - np.log1p(-o)


# ------------------------------------------------------------------------------------------
# Cameras
# ------------------------------------------------------------------------------------------

PINHOLE, FISHEYE = 0, 1


def look_at_basis(pos, target, up=(0.0, 1.0, 0.0)):
    """Orthonormal (right, up, forward) for a camera at pos looking at target."""
    pos = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    upw = np.asarray(up, dtype=np.float64)
    if abs(float(np.dot(fwd, upw))) > 0.999:
        upw = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    right = np.cross(fwd, upw)
    right /= np.linalg.norm(right)
    up_c = np.cross(right, fwd)
    return right, up_c, fwd


def pinhole_camera(width, height, pos, target=(0.0, 0.0, 0.0), fov_y_deg=60.0, t_near=0.0,
                   t_far=math.inf, up=(0.0, 1.0, 0.0)) -> dict:
    right, up_c, fwd = look_at_basis(pos, target, up)
    return dict(type=PINHOLE, width=int(width), height=int(height), pos=tuple(map(float, pos)),
                right=tuple(right), up=tuple(up_c), forward=tuple(fwd), fov=math.radians(fov_y_deg),
                t_near=float(t_near), t_far=float(t_far))


def fisheye_camera(width, height, pos, forward_dir, theta_half_width_deg=90.0, t_near=0.0,
                   t_far=math.inf, up=(0.0, 1.0, 0.0)) -> dict:
    """Equidistant fisheye: angle from the axis grows linearly with pixel radius and
    reaches theta_half_width at half the image width."""
    target = np.asarray(pos, dtype=np.float64) + np.asarray(forward_dir, dtype=np.float64)
    right, up_c, fwd = look_at_basis(pos, target, up)
    return dict(type=FISHEYE, width=int(width), height=int(height), pos=tuple(map(float, pos)),
                right=tuple(right), up=tuple(up_c), forward=tuple(fwd),
                fov=math.radians(theta_half_width_deg), t_near=float(t_near), t_far=float(t_far))


def crop_rays_index(width: int, x0: int, y0: int, w: int, h: int) -> np.ndarray:
    """Row-major pixel indices of a w x h crop whose top-left pixel is (x0, y0)."""
    ys, xs = np.meshgrid(np.arange(y0, y0 + h), np.arange(x0, x0 + w), indexing="ij")
    return (ys * width + xs).reshape(-1)


# ------------------------------------------------------------------------------------------
# Scenes
# ------------------------------------------------------------------------------------------

def tiny_scene(seed: int = 0, n: int = 1000) -> GaussianParams:
    """1,000 Gaussians: means U[-1,1]^3, log-scales U[-4.5,-2.5] per axis, uniformly random
    unit quaternions, logits N(0,1), SH degree 0 with colour U[0,1]^3."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    log_scales = rng.uniform(-4.5, -2.5, (n, 3))
    quats = _normalize(rng.standard_normal((n, 4)))
    logits = rng.standard_normal(n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh = ((rgb - 0.5) * TWO_SQRT_PI).reshape(n, 1, 3)
    return GaussianParams(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), 0,
                          dict(kind="tiny", seed=seed))


def _quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    aw, ax, ay, az = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def _quat_z_to(normal: np.ndarray, twist: np.ndarray) -> np.ndarray:
    """Quaternion whose rotation takes local +z to `normal`, after a twist about +z."""
    nz = np.clip(normal[:, 2], -1.0, 1.0)
    axis = np.stack([-normal[:, 1], normal[:, 0], np.zeros_like(nz)], axis=-1)   # z x n
    s = np.linalg.norm(axis, axis=-1)
    ang = np.arctan2(s, nz)
    safe = s > 1e-12
    axis_n = np.where(safe[:, None], axis / np.where(safe, s, 1.0)[:, None], np.array([1.0, 0.0, 0.0]))
    q_align = np.concatenate([np.cos(0.5 * ang)[:, None], np.sin(0.5 * ang)[:, None] * axis_n], axis=-1)
    q_twist = np.stack([np.cos(0.5 * twist), np.zeros_like(twist), np.zeros_like(twist), np.sin(0.5 * twist)],
                       axis=-1)
    return _normalize(_quat_mul(q_align, q_twist))


def _random_unit(rng, n) -> np.ndarray:
    return _normalize(rng.standard_normal((n, 3)))


def _surface_gaussians(rng, points, normals, sh_degree, noise=0.01):
    """Gaussians lying on surfaces: anisotropic log-normal tangent scales, the flattest axis
    along the surface normal with axis ratio log-uniform in [1, 100], opacity Beta(.5,.5)."""
    n = points.shape[0]
    means = points + rng.normal(0.0, noise, (n, 3))
    st = np.exp(rng.normal(math.log(0.01), 0.3, (n, 2)))
    ratio = np.exp(rng.uniform(0.0, math.log(100.0), n))
    sn = st.min(axis=1) / ratio
    log_scales = np.log(np.concatenate([st, sn[:, None]], axis=1))
    quats = _quat_z_to(normals, rng.uniform(0.0, 2.0 * math.pi, n))
    o = np.clip(rng.beta(0.5, 0.5, n), 1e-6, 1.0 - 1e-6)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.3, (n, K, 3))
    return means, log_scales, quats, _logit(o), sh


def surface_scene(n: int = 1_000_000, seed: int = 1, n_spheres: int = 100, n_patches: int = 100,
                  sh_degree: int = 3, extent: float = 2.0) -> GaussianParams:
    """Gaussians sampled on 100 noisy spheres (r ~ U[0.1,0.6]) and 100 square patches
    (side ~ U[0.3,1.5]) with centres in [-extent, extent]^3; counts proportional to area."""
    rng = np.random.default_rng(seed)
    sph_c = rng.uniform(-extent, extent, (n_spheres, 3))
    sph_r = rng.uniform(0.1, 0.6, n_spheres)
    pat_c = rng.uniform(-extent, extent, (n_patches, 3))
    pat_side = rng.uniform(0.3, 1.5, n_patches)
    pat_n = _random_unit(rng, n_patches)
    tmp = _random_unit(rng, n_patches)
    pat_u = _normalize(np.cross(pat_n, tmp))
    pat_v = np.cross(pat_n, pat_u)
    areas = np.concatenate([4.0 * math.pi * sph_r ** 2, pat_side ** 2])
    counts = rng.multinomial(n, areas / areas.sum())
    sid = np.repeat(np.arange(n_spheres + n_patches), counts)
    is_sph = sid < n_spheres
    pts = np.empty((n, 3)); nrm = np.empty((n, 3))
    ns = int(is_sph.sum())
    u = _random_unit(rng, ns)
    si = sid[is_sph]
    pts[is_sph] = sph_c[si] + sph_r[si, None] * u
    nrm[is_sph] = u
    pi_ = sid[~is_sph] - n_spheres
    npat = pi_.shape[0]
    ab = rng.uniform(-0.5, 0.5, (npat, 2)) * pat_side[pi_, None]
    pts[~is_sph] = pat_c[pi_] + ab[:, :1] * pat_u[pi_] + ab[:, 1:] * pat_v[pi_]
    nrm[~is_sph] = pat_n[pi_]
    perm = rng.permutation(n)
    pts, nrm = pts[perm], nrm[perm]
    means, log_scales, quats, logits, sh = _surface_gaussians(rng, pts, nrm, sh_degree)
    return GaussianParams(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), sh_degree,
                          dict(kind="surface", seed=seed, n_spheres=n_spheres, n_patches=n_patches))


def outdoor_scene(n: int = 6_000_000, seed: int = 2, size: float = 100.0, n_clusters: int = 500,
                  sh_degree: int = 3) -> GaussianParams:
    """Half the Gaussians on a size x size ground plane (y = 0), half in clusters (blobs or
    spherical shells, radii log-uniform in [0.2, 5]) scattered over it. Base scales span
    three decades, [0.005, 5] m, log-normally distributed (median 3 cm, sigma of ln 1.0, as
    trained scenes put most Gaussians in the centimetre range with a long tail); anisotropy
    as on surfaces."""
    rng = np.random.default_rng(seed)
    n_ground = n // 2
    n_cl = n - n_ground
    g_pts = np.stack([rng.uniform(-size / 2, size / 2, n_ground), np.zeros(n_ground),
                      rng.uniform(-size / 2, size / 2, n_ground)], axis=1)
    g_nrm = np.tile(np.array([0.0, 1.0, 0.0]), (n_ground, 1))
    c_center = np.stack([rng.uniform(-size / 2, size / 2, n_clusters), np.zeros(n_clusters),
                         rng.uniform(-size / 2, size / 2, n_clusters)], axis=1)
    c_rad = np.exp(rng.uniform(math.log(0.2), math.log(5.0), n_clusters))
    c_center[:, 1] = c_rad
    c_shell = rng.uniform(size=n_clusters) < 0.5
    cid = rng.integers(0, n_clusters, n_cl)
    u = _random_unit(rng, n_cl)
    rad = np.where(c_shell[cid], c_rad[cid], c_rad[cid] * np.abs(rng.normal(0.0, 0.5, n_cl)))
    c_pts = c_center[cid] + rad[:, None] * u
    pts = np.concatenate([g_pts, c_pts])
    nrm = np.concatenate([g_nrm, u])
    base = np.clip(np.exp(rng.normal(math.log(0.03), 1.0, n)), 0.005, 5.0)
    means, log_scales, quats, logits, sh = _surface_gaussians(rng, pts, nrm, sh_degree, noise=0.0)
    log_scales = log_scales - math.log(0.01) + np.log(base)[:, None]
    return GaussianParams(_f32(means), _f32(log_scales), _f32(quats), _f32(logits), _f32(sh), sh_degree,
                          dict(kind="outdoor", seed=seed, size=size))


def perturb(g: GaussianParams, sigma: float, seed: int) -> GaussianParams:
    """Every raw parameter plus N(0, sigma^2) noise."""
    rng = np.random.default_rng(seed)
    arrs = [_f32(a + rng.normal(0.0, sigma, a.shape)) for a in g.arrays()]
    return GaussianParams(*arrs, g.sh_degree, dict(g.meta, perturbed=sigma))


# ------------------------------------------------------------------------------------------
# Serving request stream
# ------------------------------------------------------------------------------------------

SERVE_RESOLUTIONS = ((256, 256), (512, 512), (1280, 720), (1920, 1080))


def request_stream(n_requests: int = 2000, rate_hz: float = 200.0, n_scenes: int = 4, seed: int = 4,
                   resolutions=SERVE_RESOLUTIONS, radius=(3.0, 10.0), fov_y_deg=60.0):
    """Poisson arrivals; resolution uniform over `resolutions`; camera direction uniform on
    the sphere at a radius uniform in `radius`, looking at the origin; scene uniform."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    res_i = rng.integers(0, len(resolutions), n_requests)
    dirs = _random_unit(rng, n_requests)
    rads = rng.uniform(radius[0], radius[1], n_requests)
    scenes = rng.integers(0, n_scenes, n_requests)
    reqs = []
    for j in range(n_requests):
        w, h = resolutions[res_i[j]]
        pos = dirs[j] * rads[j]
        reqs.append(dict(arrival=float(arrivals[j]), scene=int(scenes[j]),
                         camera=pinhole_camera(w, h, pos, (0.0, 0.0, 0.0), fov_y_deg), tag=j))
    return reqs


# ------------------------------------------------------------------------------------------
# The five workloads
# ------------------------------------------------------------------------------------------

def config_tiny():
    """1,000 Gaussians, one 64x64 pinhole camera at (0,0,-3), 60 degree FoV, k = 8, seed 0."""
    g = tiny_scene(seed=0)
    cam = pinhole_camera(64, 64, (0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 60.0)
    return g, cam, dict(k=8, alpha_min=0.01, T_min=1e-3)


def config_surface(n: int = 1_000_000, width: int = 1920, height: int = 1080):
    """1M surface-like Gaussians, SH degree 3, 1920x1080 pinhole at (0,0,-4), k = 16, seed 1."""
    g = surface_scene(n=n, seed=1)
    cam = pinhole_camera(width, height, (0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 60.0)
    return g, cam, dict(k=16, alpha_min=0.01, T_min=1e-3)


def config_differentiable(n: int = 262_144, width: int = 800, height: int = 800):
    """256K surface-like Gaussians, 800x800 pinhole; the target image is rendered from the
    same scene with every raw parameter perturbed by N(0, 0.01^2); seed 3."""
    g = surface_scene(n=n, seed=3)
    target = perturb(g, 0.01, seed=103)
    cam = pinhole_camera(width, height, (0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 60.0)
    return g, target, cam, dict(k=16, alpha_min=0.01, T_min=1e-3)


def config_serving(sizes=(500_000, 1_000_000, 2_000_000, 3_000_000), n_requests: int = 2000):
    """Four resident surface-like scenes and a 200 req/s Poisson request stream; seed 4."""
    scenes = [surface_scene(n=s, seed=40 + i) for i, s in enumerate(sizes)]
    reqs = request_stream(n_requests=n_requests, rate_hz=200.0, n_scenes=len(sizes), seed=4)
    return scenes, reqs, dict(k=16, alpha_min=0.01, T_min=1e-3)


def serving_stream_at(rate_hz: float, n_requests: int = 2000, n_scenes: int = 4):
    """The serving configuration's request stream (same seed, resolutions and poses) with
    Poisson arrivals at another rate: the views are those of the 200 req/s stream, only the
    gaps between arrivals scale by 200 / rate_hz."""
    reqs = request_stream(n_requests=n_requests, rate_hz=200.0, n_scenes=n_scenes, seed=4)
    for r in reqs:
        r["arrival"] *= 200.0 / rate_hz
    return reqs


def outdoor_mirror(seed: int = 2, cam_pos=(0.0, 1.7, 0.0), view=(1.0, 0.0, 0.0)) -> dict:
    """A 4 x 3 m rectangular mirror at a seeded pose in front of the camera: centre 5-15 m away
    within +-30 degrees of the view direction at a height of 1.5-2.5 m, facing back towards
    the camera with a random tilt of up to 20 degrees."""
    rng = np.random.default_rng(seed + 1000)
    yaw = math.radians(rng.uniform(-30.0, 30.0))
    dist = rng.uniform(5.0, 15.0)
    v = np.asarray(view, dtype=np.float64)
    side = np.cross(v, [0.0, 1.0, 0.0])
    horiz = math.cos(yaw) * v + math.sin(yaw) * side
    center = np.asarray(cam_pos, dtype=np.float64) + dist * horiz
    center[1] = rng.uniform(1.5, 2.5)
    to_cam = np.asarray(cam_pos, dtype=np.float64) - center
    to_cam /= np.linalg.norm(to_cam)
    tilt = _random_unit(rng, 1)[0] * math.sin(math.radians(rng.uniform(0.0, 20.0)))
    normal = to_cam + tilt
    normal /= np.linalg.norm(normal)
    u = np.cross([0.0, 1.0, 0.0], normal)
    u /= np.linalg.norm(u)
    w = np.cross(normal, u)
    return dict(center=tuple(center), normal=tuple(normal), axis_u=tuple(u), axis_v=tuple(w), half_u=2.0,
                half_v=1.5, t_near_secondary=1e-3)


def outdoor_glass(seed: int = 2, cam_pos=(0.0, 1.7, 0.0), view=(1.0, 0.0, 0.0)) -> dict:
    """A glass ball (index 1.5) at a seeded place in front of the camera: radius 0.5-1.5 m,
    centre 6-12 m away within +-30 degrees of the view direction, resting 0-0.5 m above the
    ground."""
    rng = np.random.default_rng(seed + 2000)
    yaw = math.radians(rng.uniform(-30.0, 30.0))
    dist = rng.uniform(6.0, 12.0)
    radius = rng.uniform(0.5, 1.5)
    v = np.asarray(view, dtype=np.float64)
    side = np.cross(v, [0.0, 1.0, 0.0])
    center = np.asarray(cam_pos, dtype=np.float64) + dist * (math.cos(yaw) * v + math.sin(yaw) * side)
    center[1] = radius + rng.uniform(0.0, 0.5)
    return dict(center=tuple(float(x) for x in center), radius=float(radius), ior=1.5, t_near_secondary=1e-3)


def config_outdoor(n: int = 6_000_000, width: int = 1920, height: int = 1080):
    """6M-Gaussian outdoor-like scene (seed 2), equidistant fisheye at (0, 1.7, 0) looking
    along +x with 90 degrees at half the width, one mirror bounce; k = 16 and 32."""
    g = outdoor_scene(n=n, seed=2)
    cam = fisheye_camera(width, height, (0.0, 1.7, 0.0), (1.0, 0.0, 0.0), 90.0)
    return g, cam, outdoor_mirror(seed=2), dict(k=16, alpha_min=0.01, T_min=1e-3)
