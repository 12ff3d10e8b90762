"""Pins for the FP64 CPU oracle: each test checks the oracle against something other than
itself (a closed form, an independent numeric method, an invariant, the paper's worked
example) so that a plausible mistake anywhere in it fails at least one test. CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2601_20429_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Y00 = 0.5 / math.sqrt(math.pi)


def qmul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw])


def rotate(q, v):
    """Hamilton sandwich q v q*, an independent way to apply a quaternion rotation."""
    q = np.asarray(q, float) / np.linalg.norm(q)
    qc = q * np.array([1, -1, -1, -1])
    return qmul(qmul(q, np.concatenate([[0.0], v])), qc)[1:]


def make_scene(means, scales, quats, opac, colors=None, sh=None, sh_degree=0):
    means = np.atleast_2d(np.asarray(means, float))
    n = means.shape[0]
    log_scales = np.log(np.broadcast_to(np.asarray(scales, float), (n, 3)))
    quats = np.broadcast_to(np.asarray(quats, float), (n, 4))
    o = np.broadcast_to(np.asarray(opac, float), (n,))
    logits = np.log(o) - np.log1p(-o)
    if sh is None:
        colors = np.broadcast_to(np.asarray(colors, float), (n, 3))
        sh = ((colors - 0.5) / Y00).reshape(n, 1, 3)
    return O.Scene(means, log_scales, quats, logits, sh, sh_degree)


def one_ray(o, d, tn=0.0, tf=math.inf):
    return (np.array([o], float), np.array([d], float), np.array([tn]), np.array([tf]))


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("b", [0.0, 0.03, 0.11])
def test_single_isotropic_gaussian(b):
    sigma, o, c = 0.07, 0.8, np.array([0.2, 0.5, 0.9])
    S = make_scene([[0, 0, 0]], sigma, [0.3, -0.5, 0.7, 0.1], o, c)
    t, d2, alpha = S.response(0, [b, 0, -3], [0, 0, 1])
    assert t == pytest.approx(3.0, abs=1e-12)
    assert d2 == pytest.approx(b * b / sigma ** 2, rel=1e-12, abs=1e-14)
    expect_alpha = o * math.exp(-0.5 * b * b / sigma ** 2)
    assert alpha == pytest.approx(expect_alpha, rel=1e-12)
    r = S.render(one_ray([b, 0, -3], [0, 0, 1]))
    if expect_alpha >= 0.01:
        np.testing.assert_allclose(r["out"][0, :3], expect_alpha * c, rtol=1e-12)
        assert r["out"][0, 3] == pytest.approx(1 - expect_alpha, rel=1e-12)
        assert r["n_blend"][0] == 1
    else:
        assert r["n_blend"][0] == 0


def test_hit_boundary_is_alpha_min():
    sigma, o = 0.05, 0.6
    S = make_scene([[0, 0, 0]], sigma, [1, 0, 0, 0], o, [1, 1, 1])
    b_star = sigma * math.sqrt(2 * math.log(o / 0.01))
    inside = S.render(one_ray([b_star * (1 - 1e-9), 0, -3], [0, 0, 1]))
    outside = S.render(one_ray([b_star * (1 + 1e-9), 0, -3], [0, 0, 1]))
    assert inside["n_blend"][0] == 1 and outside["n_blend"][0] == 0
    assert inside["out"][0, 0] == pytest.approx(0.01, rel=1e-6)


def test_rotated_anisotropic_axis_convention():
    """45 degrees about +z turns local x to (1,1,0)/sqrt2; an offset along that direction
    must be measured against s_x (the opposite rotation convention would give s_y)."""
    sx, sy, sz = 0.3, 0.1, 0.2
    h = math.radians(22.5)
    q = [math.cos(h), 0, 0, math.sin(h)]
    S = make_scene([[0.1, 0.2, 0.3]], [sx, sy, sz], q, 0.9, [1, 1, 1])
    b = 0.05
    off = b * np.array([1, 1, 0]) / math.sqrt(2)
    t, d2, _ = S.response(0, np.array([0.1, 0.2, -2.0]) + off, [0, 0, 1])
    assert d2 == pytest.approx(b * b / sx ** 2, rel=1e-12)
    assert t == pytest.approx(2.3, rel=1e-12)


def test_t_alpha_is_the_minimiser_along_an_oblique_ray():
    """Eq. t-max-resp against a numeric minimisation of the Mahalanobis distance along the
    ray, with the local frame applied through the quaternion sandwich."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(5)
    for _ in range(20):
        mu = rng.uniform(-1, 1, 3)
        s = np.exp(rng.uniform(-3, -0.5, 3))
        q = rng.standard_normal(4)
        S = make_scene([mu], s, q, 0.7, [1, 1, 1])
        ro = rng.uniform(-3, 3, 3)
        rd = mu + rng.normal(0, 0.05, 3) - ro
        rd /= np.linalg.norm(rd)
        qc = np.asarray(q) / np.linalg.norm(q) * np.array([1, -1, -1, -1])

        def m2(t):
            v = rotate(qc, ro + t * rd - mu)     # world -> local is the inverse rotation
            return float(np.sum((v / s) ** 2))

        t0 = float(np.dot(mu - ro, rd))
        res = minimize_scalar(m2, bracket=(t0 - 1, t0, t0 + 1), tol=1e-14)
        t, d2, alpha = S.response(0, ro, rd)
        assert t == pytest.approx(res.x, rel=1e-6, abs=1e-7)
        assert d2 == pytest.approx(m2(t), rel=1e-9, abs=1e-12)
        assert d2 <= res.fun + 1e-9 * max(1.0, res.fun)
        assert alpha == pytest.approx(0.7 * math.exp(-0.5 * d2), rel=1e-12)


# ---------------------------------------------------------------- unit-sphere view (Sec. IV-A)


def test_unit_sphere_transform_matches_covariance_form():
    g = scenes.tiny_scene(seed=11, n=200)
    S = O.Scene.from_params(g)
    ex = S.export()
    rng = np.random.default_rng(1)
    checked = 0
    for i in np.nonzero(ex["valid"])[0][:60]:
        for _ in range(3):
            ro = rng.uniform(-3, 3, 3)
            rd = g.means[i].astype(float) + rng.normal(0, 0.05, 3) - ro
            rd /= np.linalg.norm(rd)
            t, d2, alpha = S.response(i, ro, rd)
            tu, D2 = S.unit_sphere(i, ro, rd)
            assert tu == pytest.approx(t, rel=1e-10, abs=1e-12)
            assert ex["kappa"][i] ** 2 * D2 == pytest.approx(d2, rel=1e-8, abs=1e-10)
            if abs(D2 - 1) > 1e-9:
                assert (D2 <= 1) == (alpha >= 0.01)
            checked += 1
    assert checked > 100


def test_unit_sphere_t_invariant_under_rescaling():
    """Scaling A (the sphere radius kappa) leaves t_alpha unchanged: shrink the opacity."""
    g = scenes.tiny_scene(seed=12, n=50)
    S1 = O.Scene.from_params(g)
    g2 = g.copy()
    g2.logits[:] = 4.0
    S2 = O.Scene.from_params(g2)
    rng = np.random.default_rng(2)
    for i in range(50):
        ro = rng.uniform(-3, 3, 3)
        rd = rng.standard_normal(3)
        t1, _ = S1.unit_sphere(i, ro, rd) if S1.export()["valid"][i] else (None, None)
        if t1 is None:
            continue
        t2, _ = S2.unit_sphere(i, ro, rd)
        assert t1 == pytest.approx(t2, rel=1e-10, abs=1e-12)


def test_aabb_bounds_the_ellipsoid_tightly():
    g = scenes.tiny_scene(seed=13, n=40)
    S = O.Scene.from_params(g)
    ex = S.export()
    th = np.linspace(0, math.pi, 181)
    ph = np.linspace(0, 2 * math.pi, 361)
    TH, PH = np.meshgrid(th, ph)
    U = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    for i in np.nonzero(ex["valid"])[0]:
        q = g.quats[i].astype(float)
        s = np.exp(g.log_scales[i].astype(float))
        k = ex["kappa"][i]
        pts = np.array([rotate(q, k * s * u) for u in U[::7]]) + g.means[i]
        lo, hi = ex["aabb"][i, :3], ex["aabb"][i, 3:]
        ext = hi - lo
        assert np.all(pts >= lo - 1e-12) and np.all(pts <= hi + 1e-12)
        assert np.all(pts.min(0) - lo < 2e-3 * ext) and np.all(hi - pts.max(0) < 2e-3 * ext)


def test_rotation_matrix_matches_quaternion_sandwich():
    g = scenes.tiny_scene(seed=14, n=30)
    g.quats[:] = np.random.default_rng(3).standard_normal((30, 4)) * 3   # not unit length
    S = O.Scene.from_params(g)
    R = S.export()["R"]
    rng = np.random.default_rng(4)
    for i in range(30):
        v = rng.standard_normal(3)
        np.testing.assert_allclose(R[i] @ v, rotate(g.quats[i].astype(float), v), atol=1e-12)
        np.testing.assert_allclose(R[i] @ R[i].T, np.eye(3), atol=1e-12)
        assert np.linalg.det(R[i]) == pytest.approx(1.0, abs=1e-12)


# ---------------------------------------------------------------- spherical harmonics


def test_sh_basis_orthonormal_on_the_sphere():
    zs, wz = np.polynomial.legendre.leggauss(24)
    nph = 48
    phis = 2 * math.pi * np.arange(nph) / nph
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        r = math.sqrt(max(0.0, 1 - z * z))
        for p in phis:
            Y = O.sh_basis(3, [r * math.cos(p), r * math.sin(p), z])
            G += np.outer(Y, Y) * w * (2 * math.pi / nph)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_addition_theorem_and_parity():
    rng = np.random.default_rng(6)
    for _ in range(50):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y = O.sh_basis(3, d)
        Ym = O.sh_basis(3, -d)
        for l in range(4):
            band = Y[l * l:(l + 1) * (l + 1)]
            assert np.sum(band ** 2) == pytest.approx((2 * l + 1) / (4 * math.pi), rel=1e-12)
            np.testing.assert_allclose(Ym[l * l:(l + 1) * (l + 1)], (-1) ** l * band, atol=1e-14)


def test_sh_colour_offset_and_clamp():
    """c = max(0, sum_k Y_k f_k + 0.5): degree-0 coefficient (c-0.5)/Y00 reproduces c, and a
    negative raw value clamps to 0."""
    S = make_scene([[0, 0, 0]], 0.05, [1, 0, 0, 0], 0.5, [0.25, -0.3, 1.0])
    r = S.render(one_ray([0, 0, -3], [0, 0, 1]))
    np.testing.assert_allclose(r["out"][0, :3], 0.5 * np.array([0.25, 0.0, 1.0]), rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- compositing (Eq. volume-render)


def test_three_gaussians_on_axis_in_depth_order():
    # nearest Gaussian has the largest id, so sorting by depth matters
    means = [[0, 0, 1.0], [0, 0, 0.5], [0, 0, 0.0]]
    ops = [0.8, 0.3, 0.5]
    cols = np.array([[0.9, 0.1, 0.1], [0.1, 0.9, 0.1], [0.1, 0.1, 0.9]])
    S = make_scene(means, 0.05, [1, 0, 0, 0], ops, cols)
    r = S.render(one_ray([0, 0, -3], [0, 0, 1]), ids_cap=4)
    a1, a2, a3 = ops[2], ops[1], ops[0]
    c1, c2, c3 = cols[2], cols[1], cols[0]
    C = a1 * c1 + (1 - a1) * a2 * c2 + (1 - a1) * (1 - a2) * a3 * c3
    np.testing.assert_allclose(r["out"][0, :3], C, rtol=1e-12)
    assert r["out"][0, 3] == pytest.approx((1 - a1) * (1 - a2) * (1 - a3), rel=1e-12)
    assert list(r["ids"][0, :3]) == [2, 1, 0]


def test_early_termination_after_the_crossing_gaussian():
    means = [[0, 0, 0.0], [0, 0, 0.5], [0, 0, 1.0]]
    ops = [0.95, 0.995, 0.5]            # second alpha clamps to 0.99; T = 0.05*0.01 < 1e-3
    cols = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    S = make_scene(means, 0.05, [1, 0, 0, 0], ops, cols)
    r = S.render(one_ray([0, 0, -3], [0, 0, 1]))
    assert r["n_blend"][0] == 2
    np.testing.assert_allclose(r["out"][0, :3], [0.95, 0.05 * 0.99, 0.0], rtol=1e-12, atol=1e-15)
    assert r["out"][0, 3] == pytest.approx(0.05 * 0.01, rel=1e-12)
    r0 = S.render(one_ray([0, 0, -3], [0, 0, 1]), params=O.make_params(T_min=0.0))
    assert r0["n_blend"][0] == 3


def test_alpha_clamp():
    S = make_scene([[0, 0, 0]], 0.05, [1, 0, 0, 0], 0.999, [1, 1, 1])
    r = S.render(one_ray([0, 0, -3], [0, 0, 1]))
    np.testing.assert_allclose(r["out"][0], [0.99, 0.99, 0.99, 0.01], rtol=1e-12)


def test_equal_depth_ties_break_by_id():
    cols = np.array([[1, 0, 0], [0, 0, 1]], float)
    S = make_scene([[0, 0, 0], [0, 0, 0]], 0.05, [1, 0, 0, 0], [0.4, 0.7], cols)
    r = S.render(one_ray([0, 0, -3], [0, 0, 1]), ids_cap=2)
    assert list(r["ids"][0]) == [0, 1]
    np.testing.assert_allclose(r["out"][0, :3], 0.4 * cols[0] + 0.6 * 0.7 * cols[1], rtol=1e-12)


def test_background_and_near_far_window():
    S = make_scene([[0, 0, 0], [0, 0, 2]], 0.05, [1, 0, 0, 0], [0.5, 0.5], [[1, 0, 0], [0, 1, 0]])
    p = O.make_params(bg=(0.0, 0.0, 1.0))
    r = S.render(one_ray([0, 0, -3], [0, 0, 1], tn=0.0, tf=4.0), params=p)
    np.testing.assert_allclose(r["out"][0], [0.5, 0, 0.5, 0.5], rtol=1e-12, atol=1e-15)
    r = S.render(one_ray([0, 0, -3], [0, 0, 1], tn=3.5, tf=math.inf), params=p)
    np.testing.assert_allclose(r["out"][0], [0, 0.5, 0.5, 0.5], rtol=1e-12, atol=1e-15)


def test_ert_error_bound_on_dense_scene():
    g = scenes.tiny_scene(seed=0, n=20000)
    cam = scenes.pinhole_camera(32, 32, (0.0, 0.0, -3.0), (0, 0, 0), 60.0)
    S = O.Scene.from_params(g)
    rays = O.camera_rays(cam)
    a = S.render(rays)
    b = S.render(rays, params=O.make_params(T_min=0.0))
    Tstop = a["out"][:, 3]
    diff = np.abs(a["out"][:, :3] - b["out"][:, :3]).max(1)
    assert np.all(diff <= Tstop * 1.0 + 1e-12)
    assert (a["n_blend"] < b["n_blend"]).sum() > 10


# ---------------------------------------------------------------- round loop (Listing 1)


@pytest.fixture(scope="module", params=["tiny", "dense"])
def tiny_rounds(request):
    if request.param == "tiny":
        g, cam, _ = scenes.config_tiny()
    else:   # enough depth complexity that most rays terminate early
        g = scenes.tiny_scene(seed=0, n=20000)
        cam = scenes.pinhole_camera(32, 32, (0.0, 0.0, -3.0), (0, 0, 0), 60.0)
    S = O.Scene.from_params(g)
    rays = O.camera_rays(cam)
    ref = S.render(rays)
    return S, rays, ref


@pytest.mark.parametrize("k", [1, 2, 3, 8, 16, 32, 4096])
@pytest.mark.parametrize("checkpoint", [True, False])
def test_rounds_equal_one_sorted_pass(tiny_rounds, k, checkpoint):
    S, rays, ref = tiny_rounds
    r = S.render_rounds(rays, k=k, checkpoint=checkpoint)
    assert np.array_equal(r["out"], ref["out"])
    assert np.array_equal(r["n_blend"], ref["n_blend"])
    assert r["stats"]["fallbacks"] == 0


@pytest.mark.parametrize("caps", [(2, -1), (-1, 1), (3, 3)])
def test_rounds_with_tiny_capacities_fall_back_exactly(tiny_rounds, caps):
    S, rays, ref = tiny_rounds
    r = S.render_rounds(rays, k=4, checkpoint=True, ckpt_cap=caps[0], evict_cap=caps[1])
    assert r["stats"]["fallbacks"] > 0
    assert np.array_equal(r["out"], ref["out"])


def test_checkpointing_removes_revisits(tiny_rounds):
    S, rays, ref = tiny_rounds
    a = S.render_rounds(rays, k=4, checkpoint=True, count_unique=True)["stats"]
    b = S.render_rounds(rays, k=4, checkpoint=False, count_unique=True)["stats"]
    assert a["nodes"] + a["leaves"] == a["unique_nodes"]       # no node is fetched twice
    assert b["nodes"] + b["leaves"] > b["unique_nodes"]        # restart revisits nodes
    assert a["nodes"] < b["nodes"]
    assert a["rounds"] == b["rounds"]


def test_worked_example_kbuffer_walkthrough():
    fx = json.load(open(os.path.join(GOLDEN, "kbuffer_walkthrough.json")))
    k = fx["k"]
    kt = np.array([e[0] for e in fx["kbuffer_before"]], float)
    kid = np.array([e[1] for e in fx["kbuffer_before"]], np.int32)
    cnt, rej = O.kbuf_insert(kt, kid, k, k, *fx["new_hit"])
    assert cnt == k and rej == (pytest.approx(fx["expect_rejected"][0]), fx["expect_rejected"][1])
    assert [[float(a), int(b)] for a, b in zip(kt, kid)] == fx["expect_kbuffer_after"]
    # Listing 1: the hit is ignored only if it is nearer than the rejected entry; here it is
    # the rejected entry itself, so it is reported and t_max becomes its t_hit
    tmax_listing = fx["new_hit"][0] if not fx["new_hit"][0] < rej[0] else math.inf
    assert tmax_listing == fx["expect_listing1_tmax_after"]
    assert kt[-1] == fx["expect_tight_tmax_after"]
    ck = [t for t in fx["node_entries_after"] if t > tmax_listing]
    assert ck == fx["expect_checkpointed_listing1"]
    # a nearer hit pushes the farthest entry (id 33) out instead
    cnt, rej = O.kbuf_insert(kt, kid, cnt, k, 2.0, 7)
    assert rej == (pytest.approx(2.85), 33)
    assert list(kid) == [12, 40, 7, 8]


# ---------------------------------------------------------------- gradients


def _fd_scene(seed=21, n=24):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.4, 0.4, (n, 3))
    log_scales = rng.uniform(-2.2, -1.2, (n, 3))
    quats = rng.standard_normal((n, 4))
    o = rng.uniform(0.15, 0.85, n)     # alpha stays below the 0.99 clamp
    logits = np.log(o) - np.log1p(-o)
    sh = rng.normal(0, 0.3, (n, 16, 3))
    return [means, log_scales, quats, logits, sh]


def test_backward_matches_central_differences():
    params = _fd_scene()
    n = params[3].shape[0]
    cam = scenes.pinhole_camera(10, 10, (0.0, 0.0, -2.5), (0, 0, 0), 40.0)
    rays = O.camera_rays(cam)
    w = np.random.default_rng(7).normal(0, 1, (rays[0].shape[0], 4))

    def run(p):
        S = O.Scene(*p, sh_degree=3)
        r = S.render(rays, ids_cap=n)
        sig = (tuple(r["n_blend"]), r["ids"].tobytes())
        return float(np.sum(w * r["out"])), sig, S

    L0, sig0, S0 = run(params)
    grads = S0.backward(rays, w)
    names = ["means", "log_scales", "quats", "logits", "sh"]
    h = 1e-6
    compared = 0
    for pi, name in enumerate(names):
        flat = params[pi].reshape(-1)
        g_an = grads[name].reshape(-1)
        scale = np.abs(g_an).max()
        for j in range(flat.size):
            pp = [a.copy() for a in params]
            pm = [a.copy() for a in params]
            pp[pi].reshape(-1)[j] += h
            pm[pi].reshape(-1)[j] -= h
            Lp, sp, _ = run(pp)
            Lm, sm, _ = run(pm)
            if sp != sig0 or sm != sig0:
                continue
            g_fd = (Lp - Lm) / (2 * h)
            assert abs(g_fd - g_an[j]) <= 1e-5 * max(abs(g_an[j]), 1e-3 * scale) + 1e-9, (name, j, g_fd, g_an[j])
            compared += 1
    assert compared > 0.9 * sum(a.size for a in params)


def test_backward_term_scale_bounds_and_single_terms():
    """The term scale of og_backward (the magnitudes an element's terms are summed from) is an
    upper bound of |g| on every element (triangle inequality), zero exactly where no term
    reaches the element, and equal to |g| for SH coefficients of a Gaussian that one ray
    blends once (one term). It is the same gradient with or without the scale."""
    params = _fd_scene()
    cam = scenes.pinhole_camera(10, 10, (0.0, 0.0, -2.5), (0, 0, 0), 40.0)
    rays = O.camera_rays(cam)
    w = np.random.default_rng(7).normal(0, 1, (rays[0].shape[0], 4))
    S = O.Scene(*params, sh_degree=3)
    g = S.backward(rays, w, term_scale=True)
    g0 = S.backward(rays, w)
    for name in ("means", "log_scales", "quats", "logits", "sh"):
        a, sc = np.abs(g[name]), g[name + "_scale"]
        np.testing.assert_allclose(g[name], g0[name], rtol=1e-9, atol=1e-12 * a.max())
        assert np.all(np.isfinite(sc))                       # alphas < 0.99, colours away from 0
        assert np.all(sc >= a * (1 - 1e-12))
        assert np.all((sc > 0) == (a > 0))
        assert sc.max() > a.max()
    one = one_ray([0.01, 0.0, -3.0], [0, 0, 1])
    S1 = make_scene([[0, 0, 0]], 0.05, [1, 0, 0, 0], 0.6, sh=np.random.default_rng(3).normal(0, 0.1, (1, 16, 3)),
                    sh_degree=3)
    g1 = S1.backward(one, np.array([[0.7, -0.4, 0.2, 0.3]]), term_scale=True)
    np.testing.assert_allclose(g1["sh_scale"], np.abs(g1["sh"]), rtol=1e-14, atol=0)
    assert np.abs(g1["sh"]).max() > 0


@pytest.mark.parametrize("offset,kink", [(0.0, True), (3e-6, True), (-3e-6, True), (1e-3, False)])
def test_backward_term_scale_marks_kinks(offset, kink):
    """A colour channel whose SH sum + 0.5 sits within 1e-5 of the clamp at 0, or an alpha
    within 1e-5 of the 0.99 clamp, marks the elements it feeds with an infinite scale: a
    lower-precision evaluation may take the other side of the kink."""
    one = one_ray([0.0, 0.0, -3.0], [0, 0, 1])
    w = np.array([[0.7, -0.4, 0.2, 0.3]])
    # colour channel 1 at raw = offset (on axis: alpha = o, colour = degree-0 coefficient)
    S = make_scene([[0, 0, 0]], 0.05, [1, 0, 0, 0], 0.6, [0.3, offset, 0.8])
    g = S.backward(one, w, term_scale=True)
    assert np.isinf(g["sh_scale"][0, 0, 1]) == kink
    assert np.isfinite(g["sh_scale"][0, 0, [0, 2]]).all() and np.isfinite(g["means_scale"]).all()
    # alpha at 0.99 + offset on the axis (alpha = o there)
    S = make_scene([[0, 0, 0]], 0.05, [1, 0, 0, 0], 0.99 + offset, [0.3, 0.5, 0.8])
    g = S.backward(one, w, term_scale=True)
    for name in ("means", "log_scales", "quats", "logits"):
        assert np.isinf(g[name + "_scale"]).all() == kink
    assert np.isfinite(g["sh_scale"]).all()


# ---------------------------------------------------------------- LBVH building blocks


def test_morton_known_codes():
    bounds = np.array([0, 0, 0, 1, 1, 1], np.float32)
    pts = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [0.75, 0, 0],
                    [0.25, 0.25, 0.25]], np.float32)
    aabb = np.concatenate([pts, pts], 1)
    codes = O.morton63(aabb, bounds)
    expect = [0, 2 ** 63 - 1, 2 ** 62, 2 ** 61, 2 ** 60, 2 ** 62 + 2 ** 59, 2 ** 59 + 2 ** 58 + 2 ** 57]
    assert [int(c) for c in codes] == expect


def _pt_boxes(pts):
    pts = np.asarray(pts, np.float32)
    return np.concatenate([pts, pts], 1)


def test_morton_sized_known_codes():
    """Hand-computed size-aware codes: a point box has size 0; the diagonal of a 3-4-0 box is
    exactly 5; a box larger than twice the bounds clamps the size to 2^16 - 2."""
    unit = np.array([0, 0, 0, 1, 1, 1], np.float32)
    codes = O.morton_sized64(_pt_boxes([[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [1, 1, 1]]), unit)
    all_xyz = sum(0xE << (4 * b) for b in range(16))
    assert [int(c) for c in codes] == [0, 2 ** 63, 2 ** 62, 2 ** 61, all_xyz]
    boxes = np.array([[0, 0, 0, 1, 0, 0], [-5, -5, -5, 5, 5, 5]], np.float32)
    codes = O.morton_sized64(boxes, unit)
    assert int(codes[0]) == 2 ** 63 + 2 ** 60                        # centroid x 0.5, diagonal 1
    assert int(codes[1]) == sum(1 << (4 * b) for b in range(1, 16))  # centroid 0, size 65534
    eight = np.array([0, 0, 0, 8, 8, 8], np.float32)
    codes = O.morton_sized64(np.array([[0, 0, 0, 3, 4, 0]], np.float32), eight)
    # centroid (1.5, 2, 0) -> q = (12288, 16384, 0); diagonal 5 -> q_s = 5 * 2^15 / 8 = 20480
    assert int(codes[0]) == 2 ** 58 + 2 ** 56 + 2 ** 55 + 2 ** 51 + 2 ** 48


def test_morton_sized_position_bits_are_the_63bit_code_prefix():
    """For point boxes the x, y, z bits of the sized code are the top 16 of the 21-bit
    quantisation (the power-of-two grids nest exactly in FP32)."""
    rng = np.random.default_rng(21)
    pts = rng.uniform(-3, 7, (5000, 3)).astype(np.float32)
    pts[:10] = pts[:10].min(0)
    pts[10:20] = pts[10:20].max(0)
    boxes = _pt_boxes(pts)
    bounds = O.centroid_bounds(boxes)
    sized = O.morton_sized64(boxes, bounds)
    m63 = O.morton63(boxes, bounds)
    for c, m in zip(sized[:2000], m63[:2000]):
        c = int(c)
        assert c & sum(1 << (4 * b) for b in range(16)) == 0          # size 0
        xyz = 0
        for b in range(16):
            xyz |= ((c >> (4 * b + 1)) & 7) << (3 * b)
        assert xyz == int(m) >> 15


def test_morton_sized_monotone_in_size_and_below_empty_marker():
    c = np.array([0.25, 0.5, 0.75], np.float32)
    h = (np.arange(1001) / 4096.0).astype(np.float32)     # exact: the centroid stays c
    boxes = np.concatenate([c - h[:, None], c + h[:, None]], 1).astype(np.float32)
    codes = O.morton_sized64(boxes, np.array([0, 0, 0, 1, 1, 1], np.float32))
    assert np.all(np.diff(codes.astype(object)) > 0)
    big = np.array([[1, 1, 1, 1, 1, 1], [-1e30, -1e30, -1e30, 1e30, 1e30, 1e30]], np.float32)
    big[0, :3] -= 1e6; big[0, 3:] += 1e6 + 2
    codes = O.morton_sized64(big, np.array([0, 0, 0, 1, 1, 1], np.float32))
    assert all(int(x) < 2 ** 64 - 1 for x in codes)


def test_centroid_bounds():
    rng = np.random.default_rng(8)
    a = rng.uniform(-5, 5, (100, 6)).astype(np.float32)
    lo = np.minimum(a[:, :3], a[:, 3:]); hi = np.maximum(a[:, :3], a[:, 3:])
    aabb = np.concatenate([lo, hi], 1)
    c = (np.float32(0.5) * (aabb[:, :3] + aabb[:, 3:])).astype(np.float32)
    np.testing.assert_array_equal(O.centroid_bounds(aabb), np.concatenate([c.min(0), c.max(0)]))


def _aug_prefix(keys, i, j):
    a = (int(keys[i]) << 32) | i
    b = (int(keys[j]) << 32) | j
    return 96 - (a ^ b).bit_length()


@pytest.mark.parametrize("n,dups", [(2, False), (3, True), (17, False), (500, True), (1000, False)])
def test_radix_tree_is_the_binary_radix_tree(n, dups):
    rng = np.random.default_rng(n)
    hi = 64 if dups else 2 ** 63
    keys = np.sort(rng.integers(0, hi, n, dtype=np.uint64))
    left, right = O.radix_tree(keys)
    child_count = {}
    rng_of = {}

    def walk(ref, a_hint=None):
        if ref & O.LEAF:
            j = ref & ~O.LEAF
            child_count[("L", j)] = child_count.get(("L", j), 0) + 1
            return j, j
        child_count[("I", ref)] = child_count.get(("I", ref), 0) + 1
        a, g = walk(int(left[ref]))
        g1, b = walk(int(right[ref]))
        assert g1 == g + 1
        common = _aug_prefix(keys, a, b)
        assert _aug_prefix(keys, a, g) > common and _aug_prefix(keys, g + 1, b) > common
        assert ref in (a, b)
        rng_of[ref] = (a, b)
        return a, b

    a, b = walk(0)
    assert (a, b) == (0, n - 1)
    assert all(v == 1 for v in child_count.values())
    assert len([1 for k_ in child_count if k_[0] == "L"]) == n
    assert len([1 for k_ in child_count if k_[0] == "I"]) == n - 1
    node_box = O.refit(left, right, np.zeros((n, 6), np.float32))
    assert node_box.shape == (n - 1, 6)


def test_refit_is_the_union_of_each_range():
    rng = np.random.default_rng(9)
    n = 300
    keys = np.sort(rng.integers(0, 2 ** 20, n, dtype=np.uint64))
    left, right = O.radix_tree(keys)
    c = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    e = rng.uniform(0, 0.1, (n, 3)).astype(np.float32)
    leaf = np.concatenate([c - e, c + e], 1)
    nodes = O.refit(left, right, leaf)

    def rng_of(ref):
        if ref & O.LEAF:
            j = ref & ~O.LEAF
            return j, j
        return rng_of(int(left[ref]))[0], rng_of(int(right[ref]))[1]

    for i in range(n - 1):
        a, b = rng_of(i)
        np.testing.assert_array_equal(nodes[i, :3], leaf[a:b + 1, :3].min(0))
        np.testing.assert_array_equal(nodes[i, 3:], leaf[a:b + 1, 3:].max(0))


# ---------------------------------------------------------------- cameras


def test_pinhole_rays_linear_in_tangent_space():
    cam = scenes.pinhole_camera(64, 48, (1.0, 2.0, -3.0), (0, 0, 0), 50.0)
    o, d, tn, tf = O.camera_rays(cam)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    R = np.array([cam["right"], cam["up"], cam["forward"]])
    loc = d @ R.T
    tx = (loc[:, 0] / loc[:, 2]).reshape(48, 64)
    ty = (loc[:, 1] / loc[:, 2]).reshape(48, 64)
    step_y = 2 * math.tan(math.radians(25)) / 48
    np.testing.assert_allclose(np.diff(ty, axis=0), -step_y, atol=1e-12)
    np.testing.assert_allclose(np.diff(tx, axis=1), step_y, atol=1e-12)   # square pixels
    np.testing.assert_allclose(tx[:, ::-1], -tx, atol=1e-12)
    np.testing.assert_allclose(ty[::-1, :], -ty, atol=1e-12)
    np.testing.assert_allclose(o, np.tile([1.0, 2.0, -3.0], (64 * 48, 1)))


def test_fisheye_angle_proportional_to_radius():
    cam = scenes.fisheye_camera(40, 30, (0, 1.7, 0), (1, 0, 0), 90.0)
    o, d, tn, tf = O.camera_rays(cam)
    ys, xs = np.meshgrid(np.arange(30) + 0.5 - 15, np.arange(40) + 0.5 - 20, indexing="ij")
    r = np.hypot(xs, ys).reshape(-1)
    ang = np.arccos(np.clip(d @ np.array(cam["forward"]), -1, 1))
    np.testing.assert_allclose(ang, r * (math.pi / 2) / 20, atol=1e-12)


# ---------------------------------------------------------------- mirror bounce


def _facing_mirror():
    return dict(center=(0.0, 0.0, 0.0), normal=(0.0, 0.0, -1.0), axis_u=(1.0, 0.0, 0.0), axis_v=(0.0, 1.0, 0.0),
                half_u=0.5, half_v=0.5, t_near_secondary=1e-4)


def test_mirror_reflects_back_through_the_same_gaussian():
    """Camera at z = -3 looking at a mirror at z = 0 facing it; one Gaussian at z = -1 on the
    axis is met by the primary (t = 2) and by the reflected ray (t = 1 from the mirror), so
    C = a c + (1 - a) a c and T = (1 - a)^2."""
    a, col = 0.6, np.array([0.9, 0.3, 0.1])
    S = make_scene([[0, 0, -1.0]], 0.02, [1, 0, 0, 0], a, col)
    cam = scenes.pinhole_camera(3, 3, (0.0, 0.0, -3.0), (0, 0, 0), 10.0)
    prim, sec, spix = O.mirror_rays(cam, _facing_mirror())
    assert list(spix) == list(range(9))                  # every pixel sees the mirror
    c = 4                                                # centre pixel: the axis ray
    assert prim[3][c] == pytest.approx(3.0)
    np.testing.assert_allclose(sec[0][c], [0, 0, 0], atol=1e-15)
    np.testing.assert_allclose(sec[1][c], [0, 0, -1], atol=1e-15)
    p = S.render(prim)["out"]
    s = S.render(sec)["out"]
    out = O.composite_bounce(p, s, spix)
    np.testing.assert_allclose(out[c, :3], a * col + (1 - a) * a * col, rtol=1e-12)
    assert out[c, 3] == pytest.approx((1 - a) ** 2, rel=1e-12)


def test_mirror_misses_outside_the_rectangle_and_keeps_background():
    m = _facing_mirror()
    m["half_u"] = m["half_v"] = 0.01
    cam = scenes.pinhole_camera(5, 5, (0.0, 0.0, -3.0), (0, 0, 0), 20.0)
    prim, sec, spix = O.mirror_rays(cam, m)
    assert list(spix) == [12]                            # only the centre pixel
    assert np.isinf(prim[3][np.arange(25) != 12]).all()
    rgbT = np.tile([0.1, 0.2, 0.3, 0.5], (25, 1))
    sec_rgbT = np.array([[0.4, 0.4, 0.4, 0.25]])
    out = O.composite_bounce(rgbT, sec_rgbT, spix, bg=(0.2, 0.2, 0.2))
    np.testing.assert_allclose(out[12], [0.1 - 0.1 + 0.2, 0.2 - 0.1 + 0.2, 0.3 - 0.1 + 0.2, 0.125])
    np.testing.assert_array_equal(out[:12], rgbT[:12])


# ---------------------------------------------------------------- glass-ball refraction


def _ball(r=1.0, ior=1.5, center=(0.0, 0.0, 0.0)):
    return dict(center=center, radius=r, ior=ior, t_near_secondary=1e-4)


def test_glass_axis_ray_passes_undeviated():
    cam = scenes.pinhole_camera(1, 1, (0.0, 0.0, -5.0), (0, 0, 0), 10.0)
    prim, sec, spix = O.secondary_rays(cam, glass=[_ball()])
    assert list(spix) == [0]
    assert prim[3][0] == pytest.approx(4.0, abs=1e-12)
    np.testing.assert_allclose(sec[0][0], [0, 0, 1], atol=1e-12)
    np.testing.assert_allclose(sec[1][0], [0, 0, 1], atol=1e-12)
    assert sec[2][0] == 1e-4 and np.isinf(sec[3][0])


def test_glass_deviation_is_the_ball_lens_formula():
    """A ray at impact parameter b leaves the ball turned by 2 (theta_i - theta_t) with
    sin theta_i = b / R and sin theta_i = n sin theta_t, in the plane of the ray and the
    centre, from a point on the sphere."""
    R, n = 1.3, 1.52
    cam = scenes.pinhole_camera(15, 15, (0.2, -0.1, -6.0), (0, 0, 0), 30.0)
    prim, sec, spix = O.secondary_rays(cam, glass=[_ball(R, n)])
    assert len(spix) > 50
    c = np.zeros(3)
    for j, p in enumerate(spix):
        o, u = prim[0][p], prim[1][p] / np.linalg.norm(prim[1][p])
        b = np.linalg.norm(np.cross(c - o, u))
        ti = math.asin(b / R)
        tt = math.asin(math.sin(ti) / n)
        w = sec[1][j]
        assert np.linalg.norm(w) == pytest.approx(1.0, abs=1e-12)
        dev = math.acos(min(1.0, float(np.dot(u, w))))
        assert dev == pytest.approx(2 * (ti - tt), abs=1e-9)
        assert abs(np.dot(w, np.cross(c - o, u))) <= 1e-9                 # coplanar
        assert np.linalg.norm(sec[0][j] - c) == pytest.approx(R, abs=1e-12)
        # the primary stops on the near surface
        hit = o + prim[3][p] * prim[1][p]
        assert np.linalg.norm(hit - c) == pytest.approx(R, abs=1e-12)


def test_glass_of_index_one_continues_the_ray():
    cam = scenes.pinhole_camera(7, 7, (0.0, 0.3, -4.0), (0, 0, 0), 25.0)
    prim, sec, spix = O.secondary_rays(cam, glass=[_ball(1.0, 1.0)])
    assert len(spix) > 10
    for j, p in enumerate(spix):
        o, d = prim[0][p], prim[1][p]
        u = d / np.linalg.norm(d)
        np.testing.assert_allclose(sec[1][j], u, atol=1e-12)
        # the exit is the far root of |o + t u| = 1
        b = np.dot(o, u)
        t_far = -b + math.sqrt(b * b - (np.dot(o, o) - 1.0))
        np.testing.assert_allclose(sec[0][j], o + t_far * u, atol=1e-12)


def test_secondary_takes_the_nearest_object_and_none_from_inside():
    cam = scenes.pinhole_camera(9, 9, (0.0, 0.0, -5.0), (0, 0, 0), 20.0)
    front = dict(_facing_mirror(), center=(0.0, 0.0, -2.0), half_u=10.0, half_v=10.0)
    prim, sec, spix = O.secondary_rays(cam, mirrors=[front], glass=[_ball()])
    assert len(spix) == 81                                              # the mirror hides the ball
    np.testing.assert_allclose(prim[3], 3.0 / prim[1][:, 2], rtol=1e-12)
    np.testing.assert_allclose(sec[1][:, 2], -prim[1][:, 2])
    back = dict(front, center=(0.0, 0.0, 3.0))
    prim, sec, spix = O.secondary_rays(cam, mirrors=[back], glass=[_ball()])
    assert len(spix) == 81
    through = prim[3] < 6.0                                             # stopped on the ball
    assert 0 < through.sum() < 81
    assert np.all(np.abs(prim[3][~through] - 8.0 / prim[1][~through, 2]) < 1e-9)
    inside = scenes.pinhole_camera(5, 5, (0.0, 0.0, 0.2), (0, 0, 1.0), 40.0)
    prim, sec, spix = O.secondary_rays(inside, glass=[_ball()])
    assert len(spix) == 0 and np.isinf(prim[3]).all()


def test_glass_shows_the_gaussian_behind_it():
    """A Gaussian on the axis behind the ball is seen through it along the undeviated axis
    ray: the pixel is the Gaussian's alpha times its colour."""
    a, col = 0.7, np.array([0.2, 0.8, 0.4])
    S = make_scene([[0, 0, 3.0]], 0.05, [1, 0, 0, 0], a, col)
    cam = scenes.pinhole_camera(1, 1, (0.0, 0.0, -5.0), (0, 0, 0), 10.0)
    prim, sec, spix = O.secondary_rays(cam, glass=[_ball()])
    p = S.render(prim)["out"]
    s = S.render(sec)["out"]
    assert p[0, 3] == 1.0                                  # nothing before the ball
    out = O.composite_bounce(p, s, spix)
    np.testing.assert_allclose(out[0, :3], a * col, rtol=1e-12)
    assert out[0, 3] == pytest.approx(1 - a, rel=1e-12)


# ---------------------------------------------------------------- multi-level instancing


def _world_scene(n=3000, seed=31):
    g = scenes.surface_scene(n=n, seed=seed, n_spheres=2, n_patches=2, extent=0.4)   # SH degree 3
    return g, O.Scene.from_params(g)


def _affine(R, c):
    return np.concatenate([np.asarray(R, float), np.asarray(c, float)[:, None]], 1).reshape(12)


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_world_identity_instance_is_the_scene():
    g, S = _world_scene()
    rays = O.camera_rays(scenes.pinhole_camera(20, 16, (0.0, 0.3, -3.0), (0, 0, 0), 20.0))
    ref = S.render(rays, ids_cap=64)
    w = O.world_render([S], [0], [_affine(np.eye(3), [0, 0, 0])], rays, ids_cap=64)
    np.testing.assert_array_equal(w["out"], ref["out"])
    np.testing.assert_array_equal(w["ids"], ref["ids"])
    assert ref["n_blend"].sum() > 100


def test_world_moves_with_its_camera():
    """Moving the object and the camera by the same rigid motion leaves the image unchanged
    (the colour is evaluated along the object-frame direction)."""
    g, S = _world_scene()
    o, d, tn, tf = O.camera_rays(scenes.pinhole_camera(18, 14, (0.2, 0.1, -3.0), (0, 0, 0), 20.0))
    ref = S.render((o, d, tn, tf), ids_cap=64)
    R, c = _rot([1.0, 2.0, -0.5], 0.9), np.array([3.0, -1.0, 7.5])
    moved = (o @ R.T + c, d @ R.T, tn, tf)
    w = O.world_render([S], [0], [_affine(R, c)], moved, ids_cap=64)
    np.testing.assert_allclose(w["out"], ref["out"], atol=1e-10)
    np.testing.assert_array_equal(w["n_blend"], ref["n_blend"])


def test_world_scaled_isotropic_gaussian_closed_form():
    """An isotropic Gaussian (sigma, opacity a) placed with uniform scale s is the Gaussian of
    width s sigma: alpha = a exp(-b^2 / (2 s^2 sigma^2)) at impact parameter b, at the foot of
    the perpendicular."""
    a, col, sig, s = 0.8, np.array([0.3, 0.6, 0.9]), 0.1, 2.5
    S = make_scene([[0, 0, 0.0]], sig, [1, 0, 0, 0], a, col)
    b = np.array([0.0, 0.1, 0.3, 0.8])                  # the hit boundary is at 0.74
    o = np.stack([b, np.zeros(4), np.full(4, -5.0)], 1)
    d = np.tile([0.0, 0.0, 1.0], (4, 1))
    w = O.world_render([S], [0], [_affine(s * np.eye(3), [0, 0, 2.0])], (o, d, np.zeros(4), np.full(4, np.inf)))
    alpha = a * np.exp(-b ** 2 / (2 * (s * sig) ** 2))
    hit = alpha >= 0.01
    np.testing.assert_allclose(w["out"][hit, :3], alpha[hit, None] * col, rtol=1e-12)
    np.testing.assert_allclose(w["out"][:, 3], np.where(hit, 1 - alpha, 1.0), rtol=1e-12)
    assert hit.sum() == 3


def test_world_overlapping_copies_blend_twice_in_id_order():
    a, col = 0.6, np.array([0.9, 0.3, 0.1])
    S = make_scene([[0, 0, 0.0]], 0.05, [1, 0, 0, 0], a, col)
    ray = (np.array([[0.0, 0.0, -3.0]]), np.array([[0.0, 0.0, 1.0]]), np.zeros(1), np.full(1, np.inf))
    I = _affine(np.eye(3), [0, 0, 0])
    w = O.world_render([S], [0, 0], [I, I], ray, ids_cap=4)
    np.testing.assert_allclose(w["out"][0, :3], a * col + (1 - a) * a * col, rtol=1e-12)
    assert w["out"][0, 3] == pytest.approx((1 - a) ** 2, rel=1e-12)
    assert list(w["ids"][0, :2]) == [0, 1]


def test_world_ids_and_images_of_separate_instances():
    g, S = _world_scene()
    g2 = scenes.tiny_scene(n=120, seed=5)
    S2 = O.Scene.from_params(g2)
    o, d, tn, tf = O.camera_rays(scenes.pinhole_camera(16, 12, (0.0, 0.0, -3.0), (0, 0, 0), 50.0))
    far = _affine(np.eye(3), [100.0, 0, 0])
    w = O.world_render([S2, S], [0, 1], [far, _affine(np.eye(3), [0, 0, 0])], (o, d, tn, tf), ids_cap=64)
    ref = S.render((o, d, tn, tf), ids_cap=64)
    np.testing.assert_array_equal(w["out"], ref["out"])
    m = ref["ids"] >= 0
    np.testing.assert_array_equal(w["ids"][m], ref["ids"][m] + 120)     # after the first instance's ids


# ---------------------------------------------------------------- locally-ordered clustering


def _cubes(xs):
    xs = np.asarray(xs, np.float32)
    return np.stack([xs, np.zeros_like(xs), np.zeros_like(xs), xs + 1, np.ones_like(xs), np.ones_like(xs)], 1)


def test_ploc_merges_mutual_nearest_pairs_first():
    """Unit cubes at x = 0, 1, 10, 11: the union of two cubes d apart has area 4 (d + 1) + 2,
    so (0, 1) and (2, 3) are mutual nearest neighbours and merge first (nodes created in that
    order), then the two pairs merge into the root."""
    left, right, it = O.ploc(_cubes([0, 1, 10, 11]), radius=3)
    L = O.LEAF
    assert it == 2
    assert list(left) == [2, L | 2, L | 0] and list(right) == [1, L | 3, L | 1]


def test_ploc_breaks_ties_to_the_lower_index():
    """Cubes at 0, 2, 4: cube 1 is equally near both others and picks cube 0; cube 2 is left
    alone for one iteration."""
    left, right, it = O.ploc(_cubes([0, 2, 4]), radius=2)
    L = O.LEAF
    assert it == 2 and list(left) == [1, L | 0] and list(right) == [L | 2, L | 1]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ploc_distance_is_the_full_surface_area(axis):
    """Each of the three face terms decides a merge. A unit cube (cluster 1) sits between
    cube A, moved 2 along `axis`, and cube B, moved 1 along both other axes. The union with A
    has extents 3 along `axis` and 1 elsewhere, area 2 (3 + 3 + 1) = 14; the union with B has
    extents 2, 2 and 1, area 2 (2 + 2 + 4) = 16; A with B is larger still. So clusters 0 and 1
    are mutual nearest and merge first. Dropping the face term of B's two moved axes (4 for B,
    1 for A) would pair B with the middle cube instead."""
    A = np.array([0, 0, 0, 1, 1, 1], np.float32)
    C = A.copy()
    B = A.copy()
    A[[axis, axis + 3]] += 2
    for a in range(3):
        if a != axis:
            B[[a, a + 3]] += 1
    left, right, it = O.ploc(np.stack([A, C, B]), radius=2)
    L = O.LEAF
    assert it == 2 and list(left) == [1, L | 0] and list(right) == [L | 2, L | 1]


def test_ploc_radius_limits_the_search():
    """With radius 1 only neighbours in order are seen: cubes at 0, 9, 10, 19 with r = 1 pair
    (1, 2) first; with r = 3 as well (the nearest pair anywhere)."""
    L = O.LEAF
    for r in (1, 3):
        left, right, it = O.ploc(_cubes([0, 9, 10, 19]), radius=r)
        assert [left[2], right[2]] == [L | 1, L | 2]       # the first node created


@pytest.mark.parametrize("n,dups", [(2, False), (3, True), (50, False), (777, True)])
def test_ploc_builds_a_valid_binary_tree(n, dups):
    rng = np.random.default_rng(n)
    c = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    if dups:
        c[n // 2:] = c[: n - n // 2]
    e = rng.uniform(0, 0.1, (n, 3)).astype(np.float32)
    boxes = np.concatenate([c - e, c + e], 1)
    left, right, it = O.ploc(boxes, radius=4)
    seen_leaf = np.zeros(n, int)
    seen_node = np.zeros(n - 1, int)
    for ch in np.concatenate([left, right]):
        if ch & O.LEAF:
            seen_leaf[int(ch) & 0x7FFFFFFF] += 1
        else:
            seen_node[ch] += 1
    assert np.all(seen_leaf == 1) and seen_node[0] == 0 and np.all(seen_node[1:] == 1)
    assert 1 <= it <= n - 1
