"""In-place scene updates (grtx_scene_update): a refit keeps the tree's topology and leaf order
and recomputes records, appearance and boxes bottom-up (the refit step of the LBVH build over
Sec. IV-A's per-Gaussian bounds); a rebuild runs the whole build again. The tree only sets the
traversal cost, so after either the image must equal, bit for bit, the image of a scene built
from scratch with the new parameters, and match the FP64 oracle's brute force."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2601_20429_gb300 import native as N  # noqa: E402
from paper_2601_20429_gb300 import render as R  # noqa: E402
from paper_2601_20429_gb300 import scenes  # noqa: E402
from tests.gpu_util import RGB_TOL, compare_hit_lists  # noqa: E402

pytestmark = pytest.mark.gpu


def _base(n=20000, seed=0):
    g = scenes.tiny_scene(seed=seed, n=n)
    g.sh = np.random.default_rng(seed + 5).normal(0, 0.3, (g.n, 16, 3)).astype(np.float32)
    g.sh_degree = 3
    return g


def _cam():
    return scenes.pinhole_camera(40, 36, (0.0, 0.0, -3.0), (0, 0, 0), 60.0)


def _moved(g, seed, sigma=0.05):
    """Every parameter moved (means by a few Gaussian widths), opacities left on the same
    side of alpha_min."""
    h = scenes.perturb(g, sigma, seed)
    thr = np.log(0.01 / 0.99)                                 # opacity logit at alpha_min
    new = g.logits + (h.logits - g.logits) * 4.0
    h.logits = np.where((new > thr) == (g.logits > thr), new, g.logits).astype(np.float32)
    return h


def _image(sc, k=16, **kw):
    r = R.render(sc, _cam(), k=k, ids_cap=256, want_n_blended=True, want_stats=True, **kw)
    torch.cuda.synchronize()
    res = {key: v.cpu().numpy() for key, v in r.items()}
    res["stats"] = N.stats_dict(r["stats"])
    assert res["stats"]["bounds_errors"] == 0         # the kernels' own index checks
    return res


def _same(a, b):
    np.testing.assert_array_equal(a["rgbT"], b["rgbT"])
    np.testing.assert_array_equal(a["ids"], b["ids"])
    np.testing.assert_array_equal(a["n_blended"], b["n_blended"])


def _fresh(g, form="sphere", **kw):
    sc = R.Scene.from_params(g, form=form, **kw)
    res = _image(sc)
    sc.close()
    return res


@pytest.mark.parametrize("form,builder", [("sphere", "ploc"), ("sphere", "lbvh"), ("ico20", "ploc")])
def test_refit_equals_fresh_build(form, builder):
    g0 = _base()
    sc = R.Scene.from_params(g0, form=form, bvh_builder=builder)
    before = sc.export()[0].cpu().numpy()
    for step in range(3):                                     # several updates in a row
        g = _moved(g0, seed=100 + step)
        assert sc.update(g.means, g.log_scales, g.quats, g.logits, g.sh) is False
        _same(_image(sc), _fresh(g, form=form, bvh_builder=builder))
    after = sc.export()[0].cpu().numpy()
    # the topology is kept (child references) while the boxes moved
    np.testing.assert_array_equal(after[:, 12:14].view(np.uint32), before[:, 12:14].view(np.uint32))
    assert not np.array_equal(after[:, :12], before[:, :12])
    sc.close()


def test_refit_matches_oracle():
    g0 = _base()
    g = _moved(g0, seed=7)
    sc = R.Scene.from_params(g0)
    sc.update(g.means, g.log_scales, g.quats, g.logits, g.sh)
    res = _image(sc)
    S = O.Scene.from_params(g)
    rays = O.camera_rays(_cam())
    ref = S.render(rays, ids_cap=256)
    bad = compare_hit_lists(S, rays, res["ids"], res["n_blended"], ref["ids"], ref["n_blend"])
    assert not bad, f"{len(bad)} rays with different blend lists, e.g. {bad[:5]}"
    err = np.abs(res["rgbT"].astype(np.float64) - ref["out"]).max(1)
    assert err.max() <= RGB_TOL or all(
        [int(x) for x in res["ids"][r, : res["n_blended"][r]]] != [int(x) for x in ref["ids"][r, : ref["n_blend"][r]]]
        for r in np.nonzero(err > RGB_TOL)[0])
    sc.close()


def test_refit_culls_leaves_and_rebuilds_on_revival():
    g0 = _base()
    g0.logits[::7] = -8.0                                     # culled at build (o < alpha_min)
    sc = R.Scene.from_params(g0)
    assert sc.info()["n_valid"] == g0.n - len(g0.logits[::7])
    # leaves dropping below alpha_min stay in the tree with empty boxes: still a refit
    g1 = _moved(g0, seed=11)
    g1.logits[::7] = -8.0
    g1.logits[3::7] = -9.0
    assert sc.update(g1.means, g1.log_scales, g1.quats, g1.logits, g1.sh) is False
    _same(_image(sc), _fresh(g1))
    # a Gaussian culled at build time comes back: the refit cannot add it and rebuilds
    g2 = _moved(g0, seed=12)
    g2.logits[::7] = -8.0
    g2.logits[7] = 2.0
    assert sc.update(g2.means, g2.log_scales, g2.quats, g2.logits, g2.sh) is True
    assert sc.info()["n_valid"] == g0.n - len(g0.logits[::7]) + 1
    _same(_image(sc), _fresh(g2))
    sc.close()


def test_refit_of_one_leaf_and_of_no_leaf():
    g0 = _base(n=5)
    g0.logits[:] = -8.0
    g0.logits[2] = 3.0
    g0.means[2] = [0.0, 0.0, 0.0]
    g0.log_scales[2] = np.log([0.3, 0.2, 0.25])
    sc = R.Scene.from_params(g0)
    assert sc.info()["n_valid"] == 1
    g1 = _moved(g0, seed=3, sigma=0.02)
    g1.logits[:] = -8.0
    g1.logits[2] = 2.5
    assert sc.update(g1.means, g1.log_scales, g1.quats, g1.logits, g1.sh) is False
    _same(_image(sc), _fresh(g1))
    g1.logits[2] = -8.0                                       # the last leaf goes below alpha_min
    assert sc.update(g1.means, g1.log_scales, g1.quats, g1.logits, g1.sh) is False
    img = _image(sc)
    _same(img, _fresh(g1))
    assert img["n_blended"].sum() == 0
    g0.logits[:] = -8.0                                       # nothing valid at build: updates rebuild
    sc2 = R.Scene.from_params(g0)
    assert sc2.info()["n_valid"] == 0
    assert sc2.update(g1.means, g1.log_scales, g1.quats, g1.logits, g1.sh) is True
    g1.logits[4] = 1.0
    assert sc2.update(g1.means, g1.log_scales, g1.quats, g1.logits, g1.sh) is True
    assert sc2.info()["n_valid"] == 1
    _same(_image(sc2), _fresh(g1))
    sc.close()
    sc2.close()


@pytest.mark.parametrize("form", ["sphere", "proxy20"])
def test_rebuild_mode_equals_fresh_build(form):
    g0 = _base(n=6000)
    g = _moved(g0, seed=21)
    sc = R.Scene.from_params(g0, form=form)
    _image(sc)                                                # grows the trace workspace
    ws = sc.info()["bytes_workspace"]
    assert sc.update(g.means, g.log_scales, g.quats, g.logits, g.sh, mode="rebuild") is True
    assert sc.info()["bytes_workspace"] == ws                 # kept across the rebuild
    _same(_image(sc), _fresh(g, form=form))
    sc.close()


def test_update_rejects_bad_input():
    g0 = _base(n=3000)
    sc = R.Scene.from_params(g0)
    proxy = R.Scene.from_params(g0, form="proxy20")
    with pytest.raises(N.GrtxError, match="number of Gaussians"):
        h = g0.subset(np.arange(2000))
        sc.update(h.means, h.log_scales, h.quats, h.logits, h.sh)
    with pytest.raises(N.GrtxError, match="SH degree"):
        N.grtx_scene_update(sc.handle, N.make_gaussians(*sc.tensors[:4], sc.tensors[4][:, :4].contiguous(), 1), 0)
    with pytest.raises(N.GrtxError, match="unknown update mode"):
        N.grtx_scene_update(sc.handle, sc._g, 7)
    with pytest.raises(N.GrtxError, match="refit needs"):
        proxy.update(g0.means, g0.log_scales, g0.quats, g0.logits, g0.sh)
    # the failed calls left both scenes as they were
    _same(_image(sc), _fresh(g0))
    _same(_image(proxy), _fresh(g0, form="proxy20"))
    sc.close()
    proxy.close()


def test_training_steps_with_a_kept_scene_give_the_same_gradients():
    """Autograd with a scene kept across steps (refit each step) against a scene built anew
    each step: same images and, up to the order of the gradient atomics, the same gradients.
    Also with the kept scene and blend lists saved for the backward (a small cap, so that
    some rays overflow theirs and replay)."""
    g0 = _base(n=4000)
    cam = scenes.pinhole_camera(24, 24, (0.0, 0.0, -3.0), (0, 0, 0), 50.0)
    target = torch.rand(24 * 24, 4, device="cuda")
    kept = R.Scene.from_params(g0, bvh_builder="lbvh")
    for step in range(3):
        g = _moved(g0, seed=40 + step, sigma=0.02)
        res = {}
        for name, opts in (("fresh", {}), ("kept", {"scene": kept}), ("saved", {"scene": kept, "save_cap": 6})):
            params = [t.requires_grad_(True) for t in R.params_to_device(g)]
            out = R.render_differentiable(*params, g.sh_degree, cam, k=8, **opts)
            loss = ((out - target) ** 2).mean()
            loss.backward()
            res[name] = (out.detach().cpu().numpy(), [p.grad.cpu().numpy() for p in params])
        np.testing.assert_array_equal(res["kept"][0], res["fresh"][0])
        for a, b in zip(res["kept"][1], res["fresh"][1]):
            np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(res["saved"][0], res["fresh"][0], rtol=0, atol=1e-6)
        for a, b in zip(res["saved"][1], res["fresh"][1]):
            np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-7)
    kept.close()


def test_memory_trim_between_scenes():
    """The library's pool keeps freed memory for the next build; trimming hands it back and
    later builds and traces work as before."""
    g0 = _base(n=6000)
    first = _fresh(g0)
    N.grtx_memory_trim(0)
    _same(_fresh(g0), first)
    N.grtx_memory_trim(1 << 30)
    with pytest.raises(N.GrtxError, match="keep_bytes"):
        N.grtx_memory_trim(-5)


@pytest.mark.parametrize("quant", [False, True])
@pytest.mark.parametrize("mode", ["refit", "rebuild"])
def test_wide_nodes_follow_an_update(mode, quant):
    """A scene built with 4-wide nodes keeps them current through a refit (collapsed again
    from the refitted binary tree) and a rebuild: the 4-wide image after the update equals
    the image of a scene built from scratch with the new parameters."""
    g = _base()
    h = _moved(g, seed=3)
    sc = R.Scene.from_params(g, bvh_width=4, bvh_quantize=quant)
    _image(sc, bvh_width=4)
    sc.update(*h.arrays(), mode=mode)
    got = _image(sc, bvh_width=4)
    fresh = R.Scene.from_params(h, bvh_width=4, bvh_quantize=quant)
    ref = _image(fresh, bvh_width=4)
    _same(got, ref)
    bin_ref = _fresh(h)
    np.testing.assert_array_equal(got["n_blended"], bin_ref["n_blended"])
    assert float(np.abs(got["rgbT"] - bin_ref["rgbT"]).max()) <= RGB_TOL
    sc.close()
    fresh.close()
