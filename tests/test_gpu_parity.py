"""GPU parity: every step of the hot path, called through the C ABI, against the FP64 oracle
on the same seeded inputs."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2601_20429_gb300 import native as N  # noqa: E402
from paper_2601_20429_gb300 import render as R  # noqa: E402
from paper_2601_20429_gb300 import scenes  # noqa: E402
from tests.gpu_util import GRAD_TERM_TOL, RGB_TOL, compare_hit_lists, rel_err  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    g, cam, cfg = scenes.config_tiny()
    S = O.Scene.from_params(g)
    rays = O.camera_rays(cam)
    ref = S.render(rays, ids_cap=64)
    return g, cam, S, rays, ref


def _dense():
    g = scenes.tiny_scene(seed=0, n=20000)
    g.sh = np.random.default_rng(5).normal(0, 0.3, (g.n, 16, 3)).astype(np.float32)
    g.sh_degree = 3
    cam = scenes.pinhole_camera(40, 36, (0.0, 0.0, -3.0), (0, 0, 0), 60.0)
    return g, cam


@pytest.fixture(scope="module")
def dense():
    g, cam = _dense()
    S = O.Scene.from_params(g)
    rays = O.camera_rays(cam)
    ref = S.render(rays, ids_cap=256)
    return g, cam, S, rays, ref


# ------------------------------------------------------------------ a1: activation / transform


def test_prep_matches_oracle():
    g = scenes.surface_scene(n=5000, seed=7)
    t = R.params_to_device(g)
    gg = N.make_gaussians(*t, g.sh_degree)
    geom = torch.empty((g.n, 16), dtype=torch.float32, device="cuda")
    aabb = torch.empty((g.n, 6), dtype=torch.float32, device="cuda")
    N.grtx_prep_gaussians(gg, 0.01, geom, aabb)
    torch.cuda.synchronize()
    ex = O.Scene.from_params(g).export()
    geom = geom.cpu().numpy().astype(np.float64)
    aabb = aabb.cpu().numpy().astype(np.float64)
    v = ex["valid"]
    A = geom[:, :12].reshape(-1, 3, 4)
    scale = np.abs(ex["A"][v, :, :3]).max(axis=(1, 2))[:, None, None]
    assert np.all(np.abs(A[v, :, :3] - ex["A"][v, :, :3]) <= 2e-5 * scale)
    np.testing.assert_array_equal(A[v, :, 3], g.means[v].astype(np.float64))     # mean, exactly
    np.testing.assert_allclose(geom[v, 12], ex["o"][v], rtol=1e-5)
    np.testing.assert_allclose(-2 * geom[v, 13] / 1.4426950408889634, ex["kappa"][v] ** 2, rtol=2e-5)
    assert np.array_equal(geom[v, 14].astype(np.float32).view(np.int32), np.nonzero(v)[0].astype(np.int32))
    ext = (ex["aabb"][v, 3:] - ex["aabb"][v, :3]).max(1, keepdims=True)
    # the GPU machine is the oracle box widened slightly (conservative), never narrower
    assert np.all(aabb[v, :3] <= ex["aabb"][v, :3] + 1e-6 * ext)
    assert np.all(aabb[v, 3:] >= ex["aabb"][v, 3:] - 1e-6 * ext)
    pad = 2e-5 * ext + 4e-6 * (1.0 + np.abs(g.means[v]).max(1, keepdims=True))     # documented widening
    assert np.all(np.abs(aabb[v] - ex["aabb"][v]) <= pad)
    assert np.all(geom[~v] == 0) and np.all(np.isinf(aabb[~v]))


# ------------------------------------------------------------------ a2/a3: LBVH building blocks


def _random_boxes(n, seed, dups=False):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-3, 5, (n, 3)).astype(np.float32)
    if dups:
        c[n // 2:] = c[: n - n // 2]
    e = rng.uniform(0, 0.2, (n, 3)).astype(np.float32)
    return np.concatenate([c - e, c + e], 1).astype(np.float32)


@pytest.mark.parametrize("kind", ["centroid", "sized"])
@pytest.mark.parametrize("n,dups", [(1, False), (2, False), (1000, False), (4097, True), (300_001, False)])
def test_morton_bit_exact(n, dups, kind):
    boxes = _random_boxes(n, n, dups)
    boxes[::97] = [np.inf, np.inf, np.inf, -np.inf, -np.inf, -np.inf]     # empty boxes
    if n > 10:
        boxes[5] = [-40, -40, -40, 40, 40, 40]                             # size clamps
        boxes[7, 3:] = boxes[7, :3]                                        # a point
    d = torch.from_numpy(boxes).cuda()
    codes = torch.empty(n, dtype=torch.int64, device="cuda")
    bounds = torch.empty(6, dtype=torch.float32, device="cuda")
    fn = N.grtx_morton_codes if kind == "centroid" else N.grtx_morton_codes_sized
    fn(d, None, codes, bounds_out=bounds)
    torch.cuda.synchronize()
    valid = np.all(boxes[:, :3] <= boxes[:, 3:], axis=1)
    ob = O.centroid_bounds(boxes[valid]) if valid.any() else np.zeros(6, np.float32)
    np.testing.assert_array_equal(bounds.cpu().numpy()[: 6] if valid.any() else ob, ob)
    oc = np.full(n, np.iinfo(np.uint64).max, dtype=np.uint64)
    if valid.any():
        oc[valid] = (O.morton63 if kind == "centroid" else O.morton_sized64)(boxes[valid], ob)
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), oc)


@pytest.mark.parametrize("n,bits", [(1, 64), (5, 64), (4096, 64), (100_000, 21), (1_000_003, 64)])
def test_sort_pairs_stable_bit_exact(n, bits):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64)
    dup = rng.integers(0, n, n // 3)
    keys[dup] = keys[(dup * 7 + 1) % n]                                   # many equal keys
    vals = np.arange(n, dtype=np.uint32)
    k = torch.from_numpy(keys.view(np.int64)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    N.grtx_sort_pairs(k, v, bits)
    torch.cuda.synchronize()
    masked = keys & np.uint64((1 << bits) - 1) if bits < 64 else keys
    order = np.argsort(masked, kind="stable")
    assert np.array_equal(v.cpu().numpy().view(np.uint32), order.astype(np.uint32))
    assert np.array_equal(k.cpu().numpy().view(np.uint64), keys[order])


@pytest.mark.parametrize("n,dups", [(2, False), (3, True), (1000, False), (65_537, True)])
def test_radix_tree_and_refit_bit_exact(n, dups):
    rng = np.random.default_rng(n + 1)
    keys = np.sort(rng.integers(0, 64 if dups else 2 ** 63, n, dtype=np.uint64))
    kd = torch.from_numpy(keys.view(np.int64)).cuda()
    left = torch.empty(n - 1, dtype=torch.int32, device="cuda")
    right = torch.empty(n - 1, dtype=torch.int32, device="cuda")
    parent = torch.empty(2 * n - 1, dtype=torch.int32, device="cuda")
    N.grtx_radix_tree(kd, left, right, parent)
    boxes = _random_boxes(n, n + 2)
    lb = torch.from_numpy(boxes).cuda()
    nb = torch.empty((n - 1, 6), dtype=torch.float32, device="cuda")
    cnt = torch.empty(n - 1, dtype=torch.int32, device="cuda")
    N.grtx_refit(left, right, parent, lb, nb, cnt)
    torch.cuda.synchronize()
    ol, orr = O.radix_tree(keys)
    assert np.array_equal(left.cpu().numpy().view(np.uint32), ol)
    assert np.array_equal(right.cpu().numpy().view(np.uint32), orr)
    assert np.array_equal(nb.cpu().numpy(), O.refit(ol, orr, boxes))
    par = parent.cpu().numpy().view(np.uint32)
    assert par[0] == 0xFFFFFFFF
    for i in range(n - 1):
        for c in (ol[i], orr[i]):
            j = (n - 1 + (c & 0x7FFFFFFF)) if c & 0x80000000 else c
            assert par[j] == i


@pytest.mark.parametrize("n,dups", [(2, False), (3, True), (1000, False), (65_537, True), (400_001, False)])
def test_ploc_tree_bit_exact(n, dups):
    """The clustering tree (topology and node numbering) equals the oracle's, and refit over
    it gives the oracle's boxes."""
    boxes = _random_boxes(n, n + 5, dups)
    order = np.argsort(O.morton_sized64(boxes, O.centroid_bounds(boxes)), kind="stable")
    boxes = np.ascontiguousarray(boxes[order])
    d = torch.from_numpy(boxes).cuda()
    left = torch.empty(n - 1, dtype=torch.int32, device="cuda")
    right = torch.empty(n - 1, dtype=torch.int32, device="cuda")
    parent = torch.empty(2 * n - 1, dtype=torch.int32, device="cuda")
    it = N.grtx_ploc_tree(d, left, right, parent)
    torch.cuda.synchronize()
    ol, orr, oit = O.ploc(boxes, radius=16)
    assert it == oit
    np.testing.assert_array_equal(left.cpu().numpy().view(np.uint32), ol)
    np.testing.assert_array_equal(right.cpu().numpy().view(np.uint32), orr)
    par = parent.cpu().numpy().view(np.uint32)
    assert par[0] == 0xFFFFFFFF
    for i in range(0, n - 1, max(1, (n - 1) // 2000)):
        for c in (ol[i], orr[i]):
            j = (n - 1 + (int(c) & 0x7FFFFFFF)) if c & 0x80000000 else int(c)
            assert par[j] == i
    if n >= 1000:
        node_aabb = torch.empty((n - 1, 6), dtype=torch.float32, device="cuda")
        cnt = torch.empty(n - 1, dtype=torch.int32, device="cuda")
        N.grtx_refit(left, right, parent, d, node_aabb, cnt)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(node_aabb.cpu().numpy(), O.refit(ol, orr, boxes))


@pytest.mark.parametrize("bvh_builder", ["ploc", "lbvh"])
@pytest.mark.parametrize("bvh_codes", ["sized", "centroid"])
def test_scene_tree_is_valid_lbvh(bvh_codes, bvh_builder):
    g = scenes.surface_scene(n=20000, seed=9)
    sc = R.Scene.from_params(g, bvh_codes=bvh_codes, bvh_builder=bvh_builder)
    info = sc.info()
    nodes, ids, codes = sc.export()
    nodes = nodes.cpu().numpy()
    ids = ids.cpu().numpy()
    codes = codes.cpu().numpy().view(np.uint64)
    valid = O.Scene.from_params(g).export()["valid"]
    assert info["n_valid"] == valid.sum() == info["n_leaves"] == info["n_nodes"] + 1
    assert np.all(np.diff(codes.astype(np.float64)) >= 0)
    assert sorted(ids.tolist()) == np.nonzero(valid)[0].tolist()
    refs = nodes[:, 12:14].copy().view(np.uint32)
    assert np.all(nodes[:, 14:16] == 0)          # no proxy slack in the sphere form
    seen_leaf = np.zeros(info["n_leaves"], int)
    seen_node = np.zeros(info["n_nodes"], int)
    for r in refs.reshape(-1):
        if r & 0x80000000:
            seen_leaf[r & 0x7FFFFFFF] += 1
        else:
            seen_node[r] += 1
    assert np.all(seen_leaf == 1) and seen_node[0] == 0 and np.all(seen_node[1:] == 1)
    # every child box nests in its parent's slot box
    box_of = {}
    for i in range(info["n_nodes"]):
        for c, off in ((refs[i, 0], 0), (refs[i, 1], 6)):
            if not c & 0x80000000:
                box_of[int(c)] = nodes[i, off:off + 6]
    for i, pb in box_of.items():
        for off in (0, 6):
            cb = nodes[i, off:off + 6]
            assert np.all(cb[:3] >= pb[:3]) and np.all(cb[3:] <= pb[3:])
    assert 0 < info["depth"] < 64


# ------------------------------------------------------------------ a4: rays


@pytest.mark.parametrize("kind", ["pinhole", "fisheye"])
def test_rays_match_oracle(kind):
    if kind == "pinhole":
        cam = scenes.pinhole_camera(37, 23, (1.0, 2.0, -3.0), (0, 0, 0), 50.0, t_near=0.1, t_far=30.0)
    else:
        cam = scenes.fisheye_camera(41, 29, (0.0, 1.7, 0.0), (1, 0, 0), 90.0)
    n = cam["width"] * cam["height"]
    o = torch.empty((n, 3), device="cuda"); d = torch.empty((n, 3), device="cuda")
    tn = torch.empty(n, device="cuda"); tf = torch.empty(n, device="cuda")
    N.grtx_generate_rays(N.make_camera(cam), o, d, tn, tf)
    torch.cuda.synchronize()
    oo, od, otn, otf = O.camera_rays(cam)
    np.testing.assert_allclose(o.cpu().numpy(), oo, atol=1e-6)
    np.testing.assert_allclose(d.cpu().numpy(), od, atol=2e-6)
    np.testing.assert_allclose(tn.cpu().numpy(), otn.astype(np.float32))
    np.testing.assert_array_equal(tf.cpu().numpy(), otf.astype(np.float32))


# ------------------------------------------------------------------ a5-a9: forward trace


def _gpu_render(g, cam, form="sphere", rays=None, bvh_width=2, bvh_quantize=False, **kw):
    sc = R.Scene.from_params(g, form=form, bvh_width=bvh_width, bvh_quantize=bvh_quantize)
    if bvh_width == 4:
        kw["bvh_width"] = 4
    out = R.render(sc, cam, rays=rays, ids_cap=kw.pop("ids_cap", 64), want_n_blended=True, want_stats=True, **kw)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = N.stats_dict(out["stats"])
    assert res["stats"]["bounds_errors"] == 0         # the kernels' own index checks
    sc.close()
    return res


def _check_image(res, ref, S, rays):
    """Pixels within RGB_TOL of the oracle, and blend lists equal up to the excused FP32/FP64
    boundary cases. A pixel may exceed RGB_TOL only where its blend list legitimately differs
    (a termination index that flips because T lands within rounding of T_min changes the
    pixel by at most T_min times one colour)."""
    bad = compare_hit_lists(S, rays, res["ids"], res["n_blended"], ref["ids"], ref["n_blend"])
    assert not bad, f"{len(bad)} rays with different hit lists, e.g. {bad[:5]}"
    err = np.abs(res["rgbT"].astype(np.float64) - ref["out"]).max(1)
    for r in np.nonzero(err > RGB_TOL)[0]:
        a = [int(x) for x in res["ids"][r, : res["n_blended"][r]]]
        b = [int(x) for x in ref["ids"][r, : ref["n_blend"][r]]]
        detail = (f"ray {r}: error {err[r]:.3g}, gpu blended {len(a)}, oracle {len(b)}, "
                  f"T gpu {res['rgbT'][r, 3]:.6g} oracle {ref['out'][r, 3]:.6g}")
        assert a != b, detail + " (same blend list)"
        assert err[r] <= 3.0 * 1e-3, detail


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("traversal", ["checkpoint", "restart"])
def test_forward_tiny_parity(tiny, k, traversal):
    g, cam, S, rays, ref = tiny
    res = _gpu_render(g, cam, k=k, traversal=traversal)
    _check_image(res, ref, S, rays)
    st = res["stats"]
    assert st["rays"] == cam["width"] * cam["height"]
    assert st["fallbacks"] == 0 and st["stack_overflow"] == 0
    assert st["blended"] == int(ref["n_blend"].sum())


@pytest.mark.parametrize("k", [4, 16])
def test_forward_dense_parity_both_traversals(dense, k):
    g, cam, S, rays, ref = dense
    a = _gpu_render(g, cam, k=k, traversal="checkpoint", ids_cap=256)
    b = _gpu_render(g, cam, k=k, traversal="restart", ids_cap=256)
    _check_image(a, ref, S, rays)
    _check_image(b, ref, S, rays)
    assert a["stats"]["nodes"] < b["stats"]["nodes"]         # resume skips the revisits
    assert a["stats"]["rounds"] == b["stats"]["rounds"]
    assert (ref["n_blend"] < ref["n_hits"]).sum() > 100       # early termination is exercised


# ------------------------------------------------------------------ 4-wide nodes (paper's wide BVH)


@pytest.mark.parametrize("quant", [False, True])
@pytest.mark.parametrize("k", [4, 16])
@pytest.mark.parametrize("traversal", ["checkpoint", "restart"])
def test_wide_nodes_parity(dense, k, traversal, quant):
    """The 4-wide collapse of the tree (bvh_width 4, float or quantised child boxes) gives the
    oracle's image and blend lists, never fetches outside the scene, and fetches fewer nodes
    than the binary tree."""
    g, cam, S, rays, ref = dense
    w = _gpu_render(g, cam, k=k, traversal=traversal, ids_cap=256, bvh_width=4, bvh_quantize=quant)
    _check_image(w, ref, S, rays)
    b = _gpu_render(g, cam, k=k, traversal=traversal, ids_cap=256)
    assert w["stats"]["fallbacks"] == 0 and w["stats"]["stack_overflow"] == 0
    assert w["stats"]["rounds"] == b["stats"]["rounds"] and w["stats"]["blended"] == b["stats"]["blended"]
    assert w["stats"]["nodes"] < b["stats"]["nodes"]
    np.testing.assert_array_equal(w["n_blended"], b["n_blended"])
    assert float(np.abs(w["rgbT"] - b["rgbT"]).max()) <= RGB_TOL


@pytest.mark.parametrize("quant", [False, True])
def test_wide_nodes_tiny_every_k(tiny, quant):
    g, cam, S, rays, ref = tiny
    for k in (1, 2, 8, 32):
        res = _gpu_render(g, cam, k=k, bvh_width=4, bvh_quantize=quant)
        _check_image(res, ref, S, rays)
        assert res["stats"]["blended"] == int(ref["n_blend"].sum())


@pytest.mark.parametrize("quant", [False, True])
def test_wide_nodes_fallbacks_are_exact(dense, quant):
    """Tiny list capacities (rays redo rounds from the root) and a short warp stack (packets
    fall back to per-ray rounds) give the same image over 4-wide nodes."""
    g, cam, S, rays, ref = dense
    a = _gpu_render(g, cam, k=4, ids_cap=256, bvh_width=4, bvh_quantize=quant, ckpt_capacity=2, evict_capacity=1)
    assert a["stats"]["fallbacks"] > 0
    _check_image(a, ref, S, rays)
    b = _gpu_render(g, cam, k=4, ids_cap=256, bvh_width=4, bvh_quantize=quant, packet_stack=2)
    _check_image(b, ref, S, rays)


def test_wide_nodes_argument_errors(dense):
    g, cam, S, rays, ref = dense
    sc = R.Scene.from_params(g)                    # binary only
    with pytest.raises(N.GrtxError) as e:
        R.render(sc, cam, k=8, bvh_width=4)
    assert e.value.status == 1 and "4-wide" in str(e.value)
    sc.close()
    with pytest.raises(N.GrtxError):
        R.Scene.from_params(g, form="proxy20", bvh_width=4)
    with pytest.raises(N.GrtxError):
        R.Scene.from_params(g, bvh_quantize=True)              # quantised boxes need bvh_width 4
    sw = R.Scene.from_params(g, bvh_width=4)
    with pytest.raises(N.GrtxError):
        R.render(sw, cam, k=8, bvh_width=4, traversal="single")
    # the other entry points trace the binary nodes of a 4-wide scene
    out = R.render(sw, cam, k=8)["rgbT"]
    out4 = R.render(sw, cam, k=8, bvh_width=4)["rgbT"]
    torch.cuda.synchronize()
    assert float((out - out4).abs().max()) <= RGB_TOL
    sw.close()


# ------------------------------------------------------------------ instanced icosphere forms


@pytest.mark.parametrize("form", ["ico20", "ico80"])
@pytest.mark.parametrize("traversal", ["checkpoint", "restart", "single"])
def test_icosphere_forms_parity(dense, form, traversal):
    """Sec. IV-A's second option: the instance BVH over a shared template mesh. The template
    only filters, the exact test decides, so the image is the definition's (oracle) and the
    sphere form's blend lists; the template traversal adds node and triangle fetches."""
    g, cam, S, rays, ref = dense
    res = _gpu_render(g, cam, form=form, k=8, traversal=traversal, ids_cap=256)
    _check_image(res, ref, S, rays)
    sph = _gpu_render(g, cam, form="sphere", k=8, traversal=traversal, ids_cap=256)
    np.testing.assert_array_equal(res["ids"], sph["ids"])
    np.testing.assert_allclose(res["rgbT"], sph["rgbT"], rtol=0, atol=1e-6)
    assert res["stats"]["rounds"] == sph["stats"]["rounds"]
    assert res["stats"]["nodes"] > sph["stats"]["nodes"] and res["stats"]["leaves"] > sph["stats"]["leaves"]
    assert res["stats"]["fallbacks"] == 0


def test_icosphere_scene_backward_equals_sphere_scene():
    g, _ = _dense()
    g = g.subset(np.arange(2000))
    cam = scenes.pinhole_camera(16, 16, (0.0, 0.0, -3.0), (0, 0, 0), 45.0)
    w = torch.from_numpy(np.random.default_rng(3).normal(0, 1, (256, 4)).astype(np.float32)).cuda()
    out = {}
    for form in ("sphere", "ico80"):
        sc = R.Scene.from_params(g, form=form)
        fwd = R.render(sc, cam, k=8)["rgbT"]
        out[form] = {k: v.cpu().numpy() for k, v in R.backward(sc, cam, fwd, w, k=8).items()}
        sc.close()
    for name in out["sphere"]:
        np.testing.assert_allclose(out["ico80"][name], out["sphere"][name], rtol=1e-5, atol=1e-6)


# ------------------------------------------------------------------ warp-packet fallback


@pytest.mark.parametrize("form,traversal", [("sphere", "checkpoint"), ("sphere", "restart"), ("sphere", "single"),
                                            ("proxy20", "checkpoint"), ("ico20", "restart")])
def test_packet_stack_overflow_falls_back_exactly(dense, form, traversal):
    """A warp whose packet would outgrow its stack traces its rays one by one: forcing that
    with a one-entry stack leaves every blend list unchanged."""
    g, cam, S, rays, ref = dense
    full = _gpu_render(g, cam, form=form, k=8, traversal=traversal, ids_cap=256)
    tiny = _gpu_render(g, cam, form=form, k=8, traversal=traversal, ids_cap=256, packet_stack=1)
    np.testing.assert_array_equal(tiny["ids"], full["ids"])
    np.testing.assert_allclose(tiny["rgbT"], full["rgbT"], rtol=0, atol=1e-6)
    if traversal != "restart":
        assert tiny["stats"]["fallbacks"] > 0
    _check_image(tiny, ref, S, rays)


# ------------------------------------------------------------------ single-round traversal


@pytest.mark.parametrize("form", ["sphere", "proxy20"])
def test_single_round_parity(dense, form):
    """Collect every hit, then sort and blend (Sec. III-C Obs. II): the definition of the
    image, so it matches the oracle, blends exactly the k-buffer rounds' lists and collects
    every hit of every ray, past the termination point too."""
    g, cam, S, rays, ref = dense
    res = _gpu_render(g, cam, form=form, traversal="single", ids_cap=256)
    _check_image(res, ref, S, rays)
    st = res["stats"]
    assert st["rounds"] == st["rays"] and st["fallbacks"] == 0
    assert st["ckpt_writes"] == 0 and st["evictions"] == 0
    assert st["blended"] == int(ref["n_blend"].sum())
    if form == "sphere":
        # every hit is collected once (up to the alpha_min boundary flips of FP32)
        assert abs(st["collected"] - int(ref["n_hits"].sum())) <= 1e-4 * int(ref["n_hits"].sum()) + 2
    else:
        assert st["collected"] >= int(ref["n_hits"].sum())       # duplicates through triangles
    # same blend lists; the colour may differ in the last bit where the compiler contracted
    # the SH polynomial differently in the two kernels
    rounds = _gpu_render(g, cam, form=form, k=8, traversal="checkpoint", ids_cap=256)
    np.testing.assert_array_equal(res["ids"], rounds["ids"])
    np.testing.assert_array_equal(res["n_blended"], rounds["n_blended"])
    np.testing.assert_allclose(res["rgbT"], rounds["rgbT"], rtol=0, atol=1e-6)


@pytest.mark.parametrize("form", ["sphere", "proxy20"])
def test_single_round_overflow_falls_back_exactly(dense, form):
    g, cam, S, rays, ref = dense
    res = _gpu_render(g, cam, form=form, traversal="single", ckpt_capacity=5, ids_cap=256)
    assert res["stats"]["fallbacks"] > 0
    _check_image(res, ref, S, rays)
    full = _gpu_render(g, cam, form=form, traversal="single", ids_cap=256)
    np.testing.assert_array_equal(res["ids"], full["ids"])
    np.testing.assert_allclose(res["rgbT"], full["rgbT"], rtol=0, atol=1e-6)


def test_single_round_rejected_where_unsupported(dense):
    g = dense[0]
    sc = R.Scene.from_params(g)
    cam = scenes.pinhole_camera(16, 16, (0.0, 0.0, -3.0), (0, 0, 0), 60.0)
    out = torch.empty((256, 4), device="cuda")
    p = N.make_params(traversal=2)
    with pytest.raises(N.GrtxError, match="traversal") as e:
        N.grtx_trace_forward_noalloc(sc.handle, N.make_camera(cam), p, out)
    assert e.value.status == 1
    from paper_2601_20429_gb300.serve import Server
    with pytest.raises(N.GrtxError, match="traversal") as e:
        Server([sc], traversal="single")
    assert e.value.status == 1
    sc.close()


@pytest.mark.parametrize("caps", [(2, 0), (0, 1), (3, 3)])
def test_forward_capacity_fallback_is_exact(dense, caps):
    g, cam, S, rays, ref = dense
    res = _gpu_render(g, cam, k=4, ckpt_capacity=caps[0], evict_capacity=caps[1], ids_cap=256)
    assert res["stats"]["fallbacks"] > 0
    _check_image(res, ref, S, rays)


@pytest.mark.parametrize("k", [4, 16])
@pytest.mark.parametrize("traversal", ["restart", "checkpoint"])
def test_forward_proxy_form_parity(dense, k, traversal):
    g, cam, S, rays, ref = dense
    res = _gpu_render(g, cam, form="proxy20", k=k, traversal=traversal, ids_cap=256)
    _check_image(res, ref, S, rays)
    assert res["stats"]["blended"] == int(ref["n_blend"].sum())


@pytest.mark.parametrize("form", ["sphere", "proxy20"])
def test_image_independent_of_bvh_codes(form):
    """The tree shape (sort key and builder) changes the cost, never the result: the same
    Gaussians in the same (t, id) order are blended with the same arithmetic, so the images are
    bitwise equal."""
    g = scenes.outdoor_scene(n=30000, seed=12, size=16.0, n_clusters=30)
    cam = scenes.fisheye_camera(72, 40, (0.0, 1.7, 0.0), (1.0, 0.0, 0.0), 90.0)
    out, nodes = {}, {}
    for codes, builder in (("sized", "ploc"), ("centroid", "ploc"), ("sized", "lbvh"), ("centroid", "lbvh")):
        sc = R.Scene.from_params(g, form=form, bvh_codes=codes, bvh_builder=builder)
        r = R.render(sc, cam, k=8, want_n_blended=True, want_stats=True)
        torch.cuda.synchronize()
        out[codes, builder] = (r["rgbT"].cpu().numpy(), r["n_blended"].cpu().numpy())
        nodes[codes, builder] = N.stats_dict(r["stats"])["nodes"]
        assert 0 < sc.info()["depth"] < 128
        sc.close()
    ref = out["sized", "ploc"]
    for key, v in out.items():
        np.testing.assert_array_equal(v[0], ref[0])
        np.testing.assert_array_equal(v[1], ref[1])
    assert ref[1].sum() > 0 and len(set(nodes.values())) == 4


def test_forward_proxy_checkpoint_fallback_is_exact(dense):
    g, cam, S, rays, ref = dense
    res = _gpu_render(g, cam, form="proxy20", k=4, traversal="checkpoint", ckpt_capacity=3, evict_capacity=2,
                      ids_cap=256)
    assert res["stats"]["fallbacks"] > 0
    _check_image(res, ref, S, rays)


@pytest.mark.parametrize("form,traversal", [("sphere", "checkpoint"), ("sphere", "restart"), ("proxy20", "checkpoint")])
def test_forward_ragged_image(form, traversal):
    """An image whose sides are not multiples of the 8x4 warp tile (ragged tiles on the right
    and bottom edges), with a fisheye camera."""
    g, _ = _dense()
    cam = scenes.fisheye_camera(37, 23, (0.0, 0.0, -3.0), (0.0, 0.0, 1.0), 40.0)
    S = O.Scene.from_params(g)
    rays = O.camera_rays(cam)
    r32 = tuple(a.astype(np.float32).astype(np.float64) for a in rays)
    ref = S.render(r32, ids_cap=256)
    trays = tuple(torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in rays)
    res = _gpu_render(g, None, form=form, rays=trays, k=8, traversal=traversal, ids_cap=256)
    _check_image(res, ref, S, r32)
    # the same camera generated in-kernel covers every pixel exactly once
    res2 = _gpu_render(g, cam, form=form, k=8, traversal=traversal, ids_cap=256)
    assert res2["stats"]["rays"] == 37 * 23
    assert np.abs(res2["rgbT"] - res["rgbT"]).max() <= 1e-3


def test_forward_explicit_rays_and_window(dense):
    g, cam, S, rays, ref = dense
    rng = np.random.default_rng(3)
    n = 700
    o = rng.uniform(-2.5, 2.5, (n, 3))
    d = rng.standard_normal((n, 3)) * rng.uniform(0.5, 2.0, (n, 1))     # not unit length
    tn = rng.uniform(0.0, 0.5, n)
    tf = tn + rng.uniform(0.5, 6.0, n)
    orays = (o, d, tn, tf)
    oref = S.render(orays, ids_cap=256)
    trays = tuple(torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in orays)
    res = _gpu_render(g, None, rays=trays, k=8, ids_cap=256)
    o32 = tuple(a.astype(np.float32).astype(np.float64) for a in orays)
    oref = S.render(o32, ids_cap=256)
    _check_image(res, oref, S, o32)


def test_forward_background_and_empty_scene():
    g = scenes.tiny_scene(seed=3, n=50)
    cam = scenes.pinhole_camera(16, 16, (0.0, 0.0, -3.0), (0, 0, 0), 60.0)
    S = O.Scene.from_params(g)
    rays = O.camera_rays(cam)
    ref = S.render(rays, params=O.make_params(bg=(0.2, 0.4, 0.6)), ids_cap=64)
    res = _gpu_render(g, cam, k=4, bg=(0.2, 0.4, 0.6))
    _check_image(res, ref, S, rays)
    g0 = g.copy()
    g0.logits[:] = -20.0                  # every opacity below alpha_min: nothing is hit
    res = _gpu_render(g0, cam, k=4, bg=(0.2, 0.4, 0.6))
    np.testing.assert_allclose(res["rgbT"], np.tile([0.2, 0.4, 0.6, 1.0], (256, 1)), atol=0)
    g1 = g.subset([int(np.argmax(g.logits))])
    S1 = O.Scene.from_params(g1)
    ref1 = S1.render(rays, ids_cap=4)
    res1 = _gpu_render(g1, cam, k=2)
    _check_image(res1, ref1, S1, rays)


@pytest.mark.slow
def test_forward_surface_full_size_sampled():
    """1M-Gaussian surface scene at 1920x1080, k = 16, through the uninstrumented kernel that
    bench.py times (no ids, counters or stats requested): 4 seeded 16x16 crops element by
    element against the oracle (brute force over every Gaussian). Then the instrumented
    kernel on the same frame: its blend lists on the crops against the oracle's, and its
    whole image against the timed kernel's."""
    g, cam, cfg = scenes.config_surface()
    sc = R.Scene.from_params(g)
    timed = R.render(sc, cam, k=16)["rgbT"]
    torch.cuda.synchronize()
    timed = timed.cpu().numpy()
    out = R.render(sc, cam, k=16, ids_cap=512, want_n_blended=True)
    torch.cuda.synchronize()
    rgbT = out["rgbT"].cpu().numpy()
    ids = out["ids"].cpu().numpy()
    nb = out["n_blended"].cpu().numpy()
    S = O.Scene.from_params(g)
    rays = O.camera_rays(cam)
    rng = np.random.default_rng(11)
    idx = np.concatenate([scenes.crop_rays_index(cam["width"], int(rng.integers(0, cam["width"] - 16)),
                                                 int(rng.integers(0, cam["height"] - 16)), 16, 16)
                          for _ in range(4)])
    sub = tuple(a[idx] for a in rays)
    ref = S.render(sub, ids_cap=512)
    err_timed = np.abs(timed[idx].astype(np.float64) - ref["out"]).max(0)
    assert err_timed.max() <= RGB_TOL, err_timed
    err = np.abs(rgbT[idx].astype(np.float64) - ref["out"]).max(0)
    assert err.max() <= RGB_TOL, err
    bad = compare_hit_lists(S, sub, ids[idx], nb[idx], ref["ids"], ref["n_blend"])
    assert not bad
    # the two instantiations differ only in the compiler's contraction of the blend arithmetic
    assert float(np.abs(timed - rgbT).max()) <= RGB_TOL
    # the same frame over the 4-wide collapse of the same tree, float and quantised child boxes
    for quant in (False, True):
        sc4 = R.Scene.from_params(g, bvh_width=4, bvh_quantize=quant)
        wide = R.render(sc4, cam, k=16, bvh_width=4)["rgbT"]
        st4 = N.stats_dict(R.render(sc4, cam, k=16, bvh_width=4, want_stats=True)["stats"])
        torch.cuda.synchronize()
        assert float(np.abs(wide.cpu().numpy() - timed).max()) <= RGB_TOL
        assert st4["bounds_errors"] == 0 and st4["fallbacks"] == 0
        sc4.close()
    assert np.all(timed[:, 3] >= 0) and np.all(timed[:, 3] <= 1) and np.isfinite(timed).all()
    assert float(timed[:, 3].min()) < 0.5        # the frame hits Gaussians
    sc.close()


# ------------------------------------------------------------------ a10: backward


def test_backward_matches_oracle_gradient():
    g, cam = _dense()
    g = g.subset(np.arange(3000))
    cam = scenes.pinhole_camera(24, 20, (0.0, 0.0, -3.0), (0, 0, 0), 45.0)
    rng = np.random.default_rng(8)
    w = rng.normal(0, 1, (cam["width"] * cam["height"], 4))
    sc = R.Scene.from_params(g)
    S = O.Scene.from_params(g)
    rays = O.camera_rays(cam)
    ref = S.backward(rays, w, term_scale=True)
    _compare_gradients_with_oracle(S, sc, cam, None, rays, w, ref, 4)


def test_autograd_function_runs_and_matches_backward():
    g, cam = _dense()
    g = g.subset(np.arange(2000))
    cam = scenes.pinhole_camera(16, 16, (0.0, 0.0, -3.0), (0, 0, 0), 45.0)
    params = [torch.from_numpy(a).cuda().requires_grad_(True) for a in g.arrays()]
    out = R.render_differentiable(*params, g.sh_degree, cam, k=8)
    w = torch.randn_like(out)
    (out * w).sum().backward()
    S = O.Scene.from_params(g)
    ref = S.backward(O.camera_rays(cam), w.cpu().numpy().astype(np.float64))
    assert rel_err(params[0].grad.cpu().numpy(), ref["means"]) <= 1e-3
    assert rel_err(params[4].grad.cpu().numpy(), ref["sh"]) <= 1e-3


@pytest.mark.slow
def test_backward_fd_cut_of_the_differentiable_scene():
    """The 256K-Gaussian differentiable scene: the FD cut is the 2,000 Gaussians with the
    largest total blend weight in the centre 32x32 crop of the 800x800 view (chosen by the
    oracle). On the cut, the oracle's analytic gradient is checked by FP64 central differences
    on a random subset of raw parameters (where the blend lists do not change), and the GPU
    gradient must match the oracle's to 1e-3 per parameter tensor."""
    g, target, cam, cfg = scenes.config_differentiable()
    o, d, tn, tf = O.camera_rays(cam)
    idx = scenes.crop_rays_index(cam["width"], 384, 384, 32, 32)
    crop = tuple(np.ascontiguousarray(a[idx].astype(np.float32).astype(np.float64)) for a in (o, d, tn, tf))
    S_full = O.Scene.from_params(g)
    ref = S_full.render(crop, ids_cap=512)
    weight = np.zeros(g.n)
    for r in range(len(idx)):
        T = 1.0
        for h in ref["ids"][r, : ref["n_blend"][r]]:
            a = min(S_full.response(int(h), crop[0][r], crop[1][r])[2], 0.99)
            weight[h] += T * a
            T *= 1 - a
    cut = np.argsort(-weight)[:2000]
    cut = cut[weight[cut] > 0]
    gc = g.subset(np.sort(cut))
    S = O.Scene.from_params(gc)
    w = np.random.default_rng(12).normal(0, 1, (len(idx), 4))
    ref_g = S.backward(crop, w, term_scale=True)
    names = {"means": "means", "log_scales": "log_scales", "quats": "quats", "opacity_logits": "logits", "sh": "sh"}
    # FP64 central differences of the oracle on a random subset of raw parameters
    rng = np.random.default_rng(13)
    base = [a.astype(np.float64) for a in gc.arrays()]

    def loss(params):
        Sx = O.Scene(*params, sh_degree=gc.sh_degree)
        r = Sx.render(crop, ids_cap=512)
        return float(np.sum(w * r["out"])), (r["n_blend"].tobytes(), r["ids"].tobytes())

    L0, sig0 = loss(base)
    h = 1e-6
    compared = 0
    for pi, key in enumerate(("means", "log_scales", "quats", "logits", "sh")):
        flat_n = base[pi].size
        for j in rng.choice(flat_n, 24, replace=False):
            pp = [a.copy() for a in base]
            pm = [a.copy() for a in base]
            pp[pi].reshape(-1)[j] += h
            pm[pi].reshape(-1)[j] -= h
            Lp, sp = loss(pp)
            Lm, sm = loss(pm)
            if sp != sig0 or sm != sig0:
                continue
            gfd = (Lp - Lm) / (2 * h)
            gan = ref_g[key].reshape(-1)[j]
            scale = np.abs(ref_g[key]).max()
            assert abs(gfd - gan) <= 1e-4 * max(abs(gan), 1e-3 * scale) + 1e-8, (key, j, gfd, gan)
            compared += 1
    assert compared >= 80
    # GPU analytic gradient on the same cut and the same FP32 rays
    sc = R.Scene.from_params(gc)
    rays = tuple(torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in crop)
    _compare_gradients_with_oracle(S, sc, None, rays, crop, w, ref_g, cfg["k"])


def _compare_gradients_with_oracle(S, sc, cam, rays_dev, rays_np, w, ref_g, k):
    """GPU gradients against the oracle's (ref_g from S.backward(..., term_scale=True)), over
    the Gaussians whose hit status is the same on both sides. A Gaussian hit on one side only
    must be a legitimate FP32/FP64 boundary case (compare_hit_lists), and is left out because
    its gradient exists on one side only.
    Per parameter tensor: relative L2 error <= 1e-3. Per element, wherever |g| > 1e-6 ||g||_inf
    and no term of the element sits at a kink of the clamps: |g_gpu - g| <= 1e-3 |g| +
    GRAD_TERM_TOL * s, with s the oracle's term scale of the element (the magnitudes its terms
    are summed from). For a sum without cancellation s is close to |g| and this is a 1e-3
    relative check; where the terms cancel, FP32 can only know the element to a multiple of
    its unit roundoff times s."""
    out = R.render(sc, cam, rays=rays_dev, k=k, ids_cap=512, want_n_blended=True)
    fwd = out["rgbT"]
    grads = R.backward(sc, cam, fwd, torch.from_numpy(w.astype(np.float32)).cuda(), rays=rays_dev, k=k)
    torch.cuda.synchronize()
    ref = S.render(rays_np, ids_cap=512)
    gid, gnb = out["ids"].cpu().numpy(), out["n_blended"].cpu().numpy()
    assert not compare_hit_lists(S, rays_np, gid, gnb, ref["ids"], ref["n_blend"])
    differ = set()
    for r in range(gnb.shape[0]):
        a = set(int(x) for x in gid[r, : gnb[r]])
        b = set(int(x) for x in ref["ids"][r, : ref["n_blend"][r]])
        differ |= a ^ b
    keep = np.ones(S.n, bool)
    keep[list(differ)] = False
    assert keep.mean() > 0.98
    names = {"means": "means", "log_scales": "log_scales", "quats": "quats", "opacity_logits": "logits", "sh": "sh"}
    for kg, ko in names.items():
        gg = grads[kg].cpu().numpy().astype(np.float64)[keep]
        go = ref_g[ko][keep]
        e = rel_err(gg, go)
        assert e <= 1e-3, (kg, e, len(differ))
        sc_ = ref_g[ko + "_scale"][keep]
        checked = (np.abs(go) > 1e-6 * np.abs(go).max()) & np.isfinite(sc_)
        assert checked.sum() >= 0.5 * (np.abs(go) > 1e-6 * np.abs(go).max()).sum()
        d = np.abs(gg - go)
        # an element no term reaches is zero on the GPU too, up to the FP32 error of a basis
        # function that vanishes exactly in FP64
        assert np.all(np.abs(gg[sc_ == 0]) <= 1e-6 * np.abs(go).max()), kg
        bad = checked & (d > 1e-3 * np.abs(go) + GRAD_TERM_TOL * sc_)
        assert not bad.any(), (kg, int(bad.sum()), int(checked.sum()),
                               [(float(gg[j]), float(go[j]), float(sc_[j])) for j in zip(*np.nonzero(bad))][:4])


# ------------------------------------------------------------------ visit log (total vs distinct fetches)


def _logged(sc, cam, stride=1, cap=4096, **kw):
    n = cam["width"] * cam["height"]
    rows = (n + stride - 1) // stride
    r = R.render(sc, cam, want_stats=True, want_n_blended=True, visit_log=(stride, rows, cap), **kw)
    torch.cuda.synchronize()
    return r, r["visits"].cpu().numpy().view(np.uint32), r["visits_n"].cpu().numpy(), N.stats_dict(r["stats"])


@pytest.mark.parametrize("form", ["sphere", "proxy20"])
def test_visit_log_counts_every_fetch_and_checkpoints_revisit_nothing(dense, form):
    """The log of every ray sums to the fetch counters. With checkpointed rounds (and no
    capacity fallback) no ray fetches a node or leaf twice (Sec. III-C); restarting from the
    root re-fetches the upper levels every round."""
    g, cam, S, rays, ref = dense
    sc = R.Scene.from_params(g, form=form)
    out = {}
    for trav in ("checkpoint", "restart"):
        r, V, n, st = _logged(sc, cam, cap=16384, k=4, traversal=trav)
        assert int(n.sum()) == st["nodes"] + st["leaves"]
        for row in range(V.shape[0]):                      # logged ids are real nodes / leaves
            ids = V[row, : min(n[row], V.shape[1])]        # (a longer trace keeps its first cap)
            inner = ids < np.uint32(0x80000000)
            assert (ids[inner] < sc.info()["n_nodes"]).all()
            assert ((ids[~inner] & 0x7FFFFFFF) < sc.info()["n_leaves"]).all()
        out[trav] = (R.visit_counts(r["visits"], r["visits_n"]), st, r["rgbT"].cpu().numpy())
    ck, rs = out["checkpoint"], out["restart"]
    np.testing.assert_allclose(ck[2], rs[2], rtol=0, atol=1e-6)
    assert rs[0]["revisit_fraction"] > 0.1
    if ck[1]["fallbacks"] == 0:
        assert ck[0]["revisit_fraction"] == 0.0 and ck[0]["fetches_per_ray"] == ck[0]["distinct_per_ray"]
    if form == "sphere":                                   # (proxy rays overflow their lists here
        assert ck[1]["fallbacks"] == 0                     #  and restart from the root)
        assert ck[0]["truncated"] == 0 and ck[0]["rays"] == cam["width"] * cam["height"]
        assert rs[1]["nodes"] + rs[1]["leaves"] > ck[1]["nodes"] + ck[1]["leaves"]
    sc.close()


def test_visit_log_samples_every_stride_th_ray(dense):
    g, cam, S, rays, ref = dense
    sc = R.Scene.from_params(g)
    _, V1, n1, _ = _logged(sc, cam, stride=1, k=8)
    _, V7, n7, _ = _logged(sc, cam, stride=7, cap=64, k=8)           # truncated rows keep the count
    np.testing.assert_array_equal(n7, n1[::7])
    for row in range(len(n7)):
        m = min(n7[row], 64)
        np.testing.assert_array_equal(V7[row, :m], V1[7 * row, :m])
    # the single-round packet path logs too: it fetches each needed node once
    r, V, n, st = _logged(sc, cam, k=8, traversal="single")
    assert int(n.sum()) == st["nodes"] + st["leaves"]
    assert R.visit_counts(r["visits"], r["visits_n"])["revisit_fraction"] == 0.0
    with pytest.raises(N.GrtxError, match="visits and visits_n"):
        rgbT = torch.empty((cam["width"] * cam["height"], 4), device="cuda")
        N.grtx_trace_forward(sc.handle, N.make_camera(cam, None), R.trace_params(), rgbT,
                             visits=torch.empty((4, 4), dtype=torch.int32, device="cuda"), visits_n=None)
    sc.close()


def test_image_shaped_ray_list_traces_in_tiles(dense):
    """A ray list with the camera's width x height is traced in the camera's 8x4 pixel tiles:
    the same image and blend lists as the camera (whose rays it holds) and as the same list
    traced as one row, and the camera's exact node counts (the same rays share each warp)."""
    g, cam, S, rays, ref = dense
    sc = R.Scene.from_params(g)
    n = cam["width"] * cam["height"]
    o, d = torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda")
    tn, tf = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    N.grtx_generate_rays(N.make_camera(cam), o, d, tn, tf)
    res = {}
    for name, c, rr in (("camera", cam, None), ("tiled", cam, (o, d, tn, tf)), ("row", None, (o, d, tn, tf))):
        r = R.render(sc, c, rays=rr, k=8, ids_cap=256, want_n_blended=True, want_stats=True)
        torch.cuda.synchronize()
        res[name] = ({key: v.cpu().numpy() for key, v in r.items() if key != "stats"}, N.stats_dict(r["stats"]))
    for name in ("tiled", "row"):
        for key in ("rgbT", "ids", "n_blended"):
            np.testing.assert_array_equal(res[name][0][key], res["camera"][0][key])
    for key in ("nodes", "leaves", "blended", "rounds", "ckpt_writes", "evictions"):
        assert res["tiled"][1][key] == res["camera"][1][key]
    assert res["row"][1]["nodes"] != res["camera"][1]["nodes"]          # other warps, other packets
    sc.close()


def test_batched_views_equal_separate_traces(dense):
    """Several views in one launch (grtx_trace_forward_batch): a camera, the same camera's
    rays as an image-shaped list, a ragged list of 777 of its rays in scrambled order and a
    second camera give, each, what grtx_trace_forward gives for it alone (to the last bit:
    the batch runs in the serving kernel, where the compiler may contract the colour
    arithmetic differently)."""
    g, cam, S, rays, ref = dense
    sc = R.Scene.from_params(g)
    n = cam["width"] * cam["height"]
    o, d = torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda")
    tn, tf = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    N.grtx_generate_rays(N.make_camera(cam), o, d, tn, tf)
    pick = torch.from_numpy(np.random.default_rng(3).permutation(n)[:777]).cuda()
    sub = (o[pick].contiguous(), d[pick].contiguous(), tn[pick].contiguous(), tf[pick].contiguous())
    cam2 = scenes.fisheye_camera(37, 23, (0.0, 0.0, -3.0), (0.0, 0.0, 1.0), 40.0)
    views = [(cam, None), (cam, (o, d, tn, tf)), (None, sub), (cam2, None)]
    for trav in ("checkpoint", "restart"):
        outs = R.render_batch(sc, views, k=8, traversal=trav)
        torch.cuda.synchronize()
        for (c, rr), got in zip(views, outs):
            alone = R.render(sc, c, rays=rr, k=8, traversal=trav)["rgbT"]
            np.testing.assert_allclose(got.cpu().numpy(), alone.cpu().numpy(), rtol=0, atol=1e-6)
    proxy = R.Scene.from_params(g.subset(np.arange(500)), form="proxy20")
    with pytest.raises(N.GrtxError, match="sphere form"):
        R.render_batch(proxy, views[:1], k=8)
    with pytest.raises(N.GrtxError, match="checkpoint or restart"):
        R.render_batch(sc, views[:1], k=8, traversal="single")
    with pytest.raises(N.GrtxError, match="n_cams"):
        R.render_batch(sc, [(cam, None)] * 65, k=8)
    proxy.close()
    sc.close()


# ------------------------------------------------------------------ saved blend lists for the backward


@pytest.mark.parametrize("traversal", ["checkpoint", "restart"])
def test_saved_blend_lists_give_the_replay_gradients(dense, traversal):
    """A forward that saves each ray's blend list gives the same image, lists that are the
    blend order of the instrumented trace, and a backward that reads them (complete lists)
    or replays the rounds (overflowed lists, cap 3 here) with the same gradients as the
    plain replay, up to the order of the atomic additions."""
    g, cam, S, rays, ref = dense
    g = g.subset(np.arange(6000))
    sc = R.Scene.from_params(g)
    inst = R.render(sc, cam, k=8, traversal=traversal, ids_cap=256, want_n_blended=True)
    plain = R.render(sc, cam, k=8, traversal=traversal)["rgbT"]
    w = torch.from_numpy(np.random.default_rng(4).normal(0, 1, (cam["width"] * cam["height"], 4))
                         .astype(np.float32)).cuda()
    replay = {key: v.cpu().numpy() for key, v in R.backward(sc, cam, plain, w, k=8, traversal=traversal).items()}
    nb = inst["n_blended"].cpu().numpy()
    leaf_ids = sc.export()[1].cpu().numpy()                     # Gaussian id of each leaf slot
    for cap in (256, 3):
        res = R.render(sc, cam, k=8, traversal=traversal, save_cap=cap)
        torch.cuda.synchronize()
        np.testing.assert_allclose(res["rgbT"].cpu().numpy(), plain.cpu().numpy(), rtol=0, atol=1e-6)
        leaves, n = (t.cpu().numpy() for t in res["saved"])
        np.testing.assert_array_equal(n, nb)
        ids = inst["ids"].cpu().numpy()
        for r in range(len(n)):
            m = min(n[r], cap)
            np.testing.assert_array_equal(leaf_ids[leaves[r, :m]], ids[r, :m])
        if cap == 3:
            assert (n > cap).mean() > 0.02 and (n <= cap).mean() > 0.02   # both paths exercised
        # the same forward image for both backwards: the saving forward is another kernel
        # instantiation, whose image may differ by an ulp, and the gradient terms at a blend
        # near full opacity divide by (1 - alpha)
        got = R.backward(sc, cam, plain, w, k=8, traversal=traversal, saved=res["saved"])
        for key, v in got.items():
            np.testing.assert_allclose(v.cpu().numpy(), replay[key], rtol=1e-4, atol=1e-6)
    sc.close()


def test_saved_blend_lists_in_autograd_and_errors(dense):
    g, cam, S, rays, ref = dense
    g = g.subset(np.arange(3000))
    target = torch.rand(cam["width"] * cam["height"], 4, device="cuda")
    grads = {}
    for save_cap in (0, 64):
        params = [t.requires_grad_(True) for t in R.params_to_device(g)]
        out = R.render_differentiable(*params, g.sh_degree, cam, k=8, save_cap=save_cap)
        ((out - target) ** 2).mean().backward()
        grads[save_cap] = [p.grad.cpu().numpy() for p in params]
    for a, b in zip(grads[64], grads[0]):
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-7)
    sc = R.Scene.from_params(g)
    proxy = R.Scene.from_params(g, form="proxy20")
    with pytest.raises(N.GrtxError, match="sphere form"):
        R.render(proxy, cam, k=8, save_cap=8)
    with pytest.raises(N.GrtxError, match="no other optional output"):
        R.render(sc, cam, k=8, save_cap=8, want_stats=True)
    with pytest.raises(N.GrtxError, match="no other optional output"):
        R.render(sc, cam, k=8, save_cap=8, traversal="single")
    sc.close()
    proxy.close()


def test_saved_list_entries_outside_the_scene_are_skipped(dense):
    """Blend lists are caller memory: an entry at or past the scene's number of valid
    Gaussians (here n_valid itself, 2^31 - 1 and 0xFFFFFFFF, as from a larger scene) is
    skipped by the backward, never read, so the gradients equal those of the same lists with
    those entries removed."""
    g, cam, S, rays, ref = dense
    g = g.subset(np.arange(4000))
    sc = R.Scene.from_params(g)
    nv = sc.info()["n_valid"]
    res = R.render(sc, cam, k=8, save_cap=128)
    leaves, n = (t.clone() for t in res["saved"])
    lv, nn = leaves.cpu().numpy(), n.cpu().numpy()
    rows = np.nonzero((nn >= 3) & (nn <= 128))[0][::3]
    assert len(rows) > 20
    bad_lv, cut_lv, cut_n = lv.copy(), lv.copy(), nn.copy()
    for q, r in enumerate(rows):
        j = q % 3                                              # first, second or third entry
        bad_lv[r, j] = (nv, 0x7FFFFFFF, -1)[q % 3]             # -1 is 0xFFFFFFFF as uint32
        cut_lv[r, j:-1] = lv[r, j + 1:]
        cut_n[r] -= 1
    w = torch.from_numpy(np.random.default_rng(9).normal(0, 1, (cam["width"] * cam["height"], 4))
                         .astype(np.float32)).cuda()
    got = {}
    for name, (a, b) in (("bad", (bad_lv, nn)), ("cut", (cut_lv, cut_n))):
        saved = (torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
        got[name] = {key: v.cpu().numpy() for key, v in
                     R.backward(sc, cam, res["rgbT"], w, k=8, saved=saved).items()}
    for key in got["cut"]:                                     # sums of float atomics in any order
        np.testing.assert_allclose(got["bad"][key], got["cut"][key], rtol=1e-4, atol=1e-6)
    sc.close()


# ------------------------------------------------------------------ zero sizes and empty windows


def test_zero_gaussians_through_every_entry_point():
    """A scene of no Gaussians: background everywhere through the plain and instrumented
    forward, saved lists, batched views and both backward paths (zero gradients), and an
    update of it; a ray list of no rays is an argument error."""
    g = scenes.tiny_scene(seed=1, n=0)
    assert g.n == 0
    cam = scenes.pinhole_camera(12, 9, (0.0, 0.0, -3.0), (0, 0, 0), 60.0)
    bg = (0.1, 0.2, 0.3)
    sc = R.Scene.from_params(g)
    assert sc.info()["n_valid"] == 0 and sc.info()["n_nodes"] == 0
    want = np.tile([0.1, 0.2, 0.3, 1.0], (cam["width"] * cam["height"], 1)).astype(np.float32)
    for kw in ({}, {"traversal": "restart"}, {"traversal": "single"}, {"ids_cap": 8, "want_stats": True}):
        r = R.render(sc, cam, k=4, bg=bg, **kw)
        np.testing.assert_allclose(r["rgbT"].cpu().numpy(), want, atol=0)
    r = R.render(sc, cam, k=4, bg=bg, save_cap=4)
    assert int(r["saved"][1].abs().sum()) == 0
    np.testing.assert_allclose(R.render_batch(sc, [(cam, None), (cam, None)], k=4, bg=bg)[1].cpu().numpy(), want, atol=0)
    dl = torch.ones((cam["width"] * cam["height"], 4), device="cuda")
    for saved in (None, r["saved"]):
        grads = R.backward(sc, cam, r["rgbT"], dl, k=4, bg=bg, saved=saved)
        assert all(v.numel() == 0 for v in grads.values())
    assert sc.update(g.means, g.log_scales, g.quats, g.logits, g.sh) is True    # nothing to refit: rebuilt
    empty = tuple(torch.empty(s, device="cuda") for s in ((0, 3), (0, 3), (0,), (0,)))
    with pytest.raises(N.GrtxError, match="camera size"):
        R.render(sc, None, rays=empty, k=4)
    sc.close()


def test_empty_and_inverted_ray_windows(dense):
    """Rays whose window (t_near, t_far] is empty or inverted see nothing, on every path."""
    g, cam, S, rays, ref = dense
    sc = R.Scene.from_params(g)
    n = cam["width"] * cam["height"]
    o, d = torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda")
    tn, tf = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    N.grtx_generate_rays(N.make_camera(cam), o, d, tn, tf)
    tn = torch.full((n,), 3.0, device="cuda")
    tf = torch.where(torch.arange(n, device="cuda") % 2 == 0, tn, tn - 1.0)   # empty, inverted
    for kw in ({}, {"traversal": "restart"}, {"traversal": "single"}, {"ids_cap": 8, "want_n_blended": True}):
        out = R.render(sc, cam, rays=(o, d, tn, tf), k=8, **kw)
        rgbT = out["rgbT"].cpu().numpy()
        np.testing.assert_array_equal(rgbT, np.tile([0.0, 0.0, 0.0, 1.0], (n, 1)).astype(np.float32))
        if "n_blended" in out:
            assert int(out["n_blended"].sum()) == 0
    sc.close()
