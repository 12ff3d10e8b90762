"""Multi-level instancing (Sec. VI "Support for Dynamic and Multi-Object Scenes"): worlds of
placed objects traced on the GPU through the C ABI against the FP64 oracle's definition
(og_world_render) on the same seeded scenes and the same FP32 placement matrices."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2601_20429_gb300 import native as N  # noqa: E402
from paper_2601_20429_gb300 import render as R  # noqa: E402
from paper_2601_20429_gb300 import scenes  # noqa: E402
from tests.gpu_util import RGB_TOL, compare_hit_lists  # noqa: E402

pytestmark = pytest.mark.gpu


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _affine(L, c):
    """3x4 row-major object-to-world map, rounded to FP32 as the GPU receives it."""
    return np.concatenate([np.asarray(L, float), np.asarray(c, float)[:, None]], 1).astype(np.float32)


class WorldResponder:
    """response(world id, ray) for the hit-list comparison: the Gaussian's oracle response
    along the ray mapped into its object's frame."""

    def __init__(self, oscenes, inst_scene, mats):
        self.S = [oscenes[i] for i in inst_scene]
        self.M = [np.asarray(m, np.float64).reshape(3, 4) for m in mats]
        self.Li = [np.linalg.inv(m[:, :3]) for m in self.M]
        self.base = np.cumsum([0] + [s.n for s in self.S])

    def response(self, wid, ro, rd):
        i = int(np.searchsorted(self.base, wid, side="right") - 1)
        oo = self.Li[i] @ (np.asarray(ro, float) - self.M[i][:, 3])
        od = self.Li[i] @ np.asarray(rd, float)
        return self.S[i].response(int(wid - self.base[i]), oo, od)


def _object(seed, n, sh3):
    g = scenes.tiny_scene(seed=seed, n=n)
    if sh3:
        g.sh = np.random.default_rng(seed + 9).normal(0, 0.3, (g.n, 16, 3)).astype(np.float32)
        g.sh_degree = 3
    return g


@pytest.fixture(scope="module")
def objects():
    g1, g2 = _object(0, 6000, True), _object(7, 2500, False)
    return [g1, g2], [O.Scene.from_params(g) for g in (g1, g2)], [R.Scene.from_params(g) for g in (g1, g2)]


def _placements():
    return [(0, _affine(np.eye(3), [0.0, 0.0, 0.0])),
            (0, _affine(0.6 * _rot([0, 1, 0.3], 0.7), [1.5, 0.2, 0.5])),
            (1, _affine(_rot([1, 0, 0], 0.5) @ np.diag([1.3, 0.7, 1.0]), [-1.2, -0.3, 0.8])),
            (0, _affine(np.eye(3), [50.0, 0.0, 0.0]))]


def _cam():
    return scenes.pinhole_camera(40, 32, (0.3, 0.2, -4.0), (0, 0, 0), 60.0)


def _check(res, ref, resp, rays):
    bad = compare_hit_lists(resp, rays, res["ids"], res["n_blended"], ref["ids"], ref["n_blend"])
    assert not bad, f"{len(bad)} rays with different blend lists, e.g. {bad[:5]}"
    err = np.abs(res["rgbT"].astype(np.float64) - ref["out"]).max(1)
    for r in np.nonzero(err > RGB_TOL)[0]:
        a = [int(x) for x in res["ids"][r, : res["n_blended"][r]]]
        b = [int(x) for x in ref["ids"][r, : ref["n_blend"][r]]]
        assert a != b and err[r] <= 3e-3, f"ray {r}: error {err[r]:.3g}"


def _gpu_world(world, cam, **kw):
    out = R.render_world(world, cam, ids_cap=kw.pop("ids_cap", 256), want_n_blended=True, want_stats=True, **kw)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = N.stats_dict(out["stats"])
    assert res["stats"]["bounds_errors"] == 0         # the kernels' own index checks
    return res


@pytest.mark.parametrize("k", [8, 16, 32])
@pytest.mark.parametrize("traversal", ["checkpoint", "restart"])
def test_world_matches_oracle(objects, k, traversal):
    gs, oscenes, gscenes = objects
    pl = _placements()
    world = R.World([(gscenes[i], M) for i, M in pl])
    cam = _cam()
    rays = O.camera_rays(cam)
    ref = O.world_render(oscenes, [i for i, _ in pl], [M for _, M in pl], rays, ids_cap=256)
    res = _gpu_world(world, cam, k=k, traversal=traversal)
    _check(res, ref, WorldResponder(oscenes, [i for i, _ in pl], [M for _, M in pl]), rays)
    st = res["stats"]
    assert st["rays"] == 40 * 32 and st["fallbacks"] == 0 and st["stack_overflow"] == 0
    assert abs(st["blended"] - int(ref["n_blend"].sum())) <= 2
    # every placed object is seen, through rotation, scale and shear
    seen = set(int(x) for x in res["ids"][res["ids"] >= 0])
    assert any(x < 6000 for x in seen) and any(6000 <= x < 12000 for x in seen)
    assert any(12000 <= x < 14500 for x in seen) and not any(x >= 14500 for x in seen)
    world.close()


def test_world_of_one_identity_instance_is_the_scene(objects):
    gs, oscenes, gscenes = objects
    world = R.World([(gscenes[0], _affine(np.eye(3), [0, 0, 0]))])
    cam = _cam()
    a = _gpu_world(world, cam, k=16)
    out = R.render(gscenes[0], cam, k=16, ids_cap=256, want_n_blended=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a["ids"], out["ids"].cpu().numpy())
    np.testing.assert_allclose(a["rgbT"], out["rgbT"].cpu().numpy(), rtol=0, atol=1e-6)
    world.close()


def test_world_checkpoints_save_revisits_and_fall_back_exactly(objects):
    gs, oscenes, gscenes = objects
    pl = _placements()
    world = R.World([(gscenes[i], M) for i, M in pl])
    cam = _cam()
    rays = O.camera_rays(cam)
    ref = O.world_render(oscenes, [i for i, _ in pl], [M for _, M in pl], rays, ids_cap=256)
    resp = WorldResponder(oscenes, [i for i, _ in pl], [M for _, M in pl])
    ck = _gpu_world(world, cam, k=4 * 2, traversal="checkpoint")
    rs = _gpu_world(world, cam, k=8, traversal="restart")
    assert ck["stats"]["nodes"] < rs["stats"]["nodes"]
    assert ck["stats"]["rounds"] == rs["stats"]["rounds"]
    tiny = _gpu_world(world, cam, k=8, traversal="checkpoint", ckpt_capacity=3, evict_capacity=2)
    assert tiny["stats"]["fallbacks"] > 0
    _check(tiny, ref, resp, rays)
    world.close()


def test_world_packet_stack_overflow_falls_back_exactly(objects):
    gs, oscenes, gscenes = objects
    pl = _placements()
    world = R.World([(gscenes[i], M) for i, M in pl])
    cam = _cam()
    a = _gpu_world(world, cam, k=16)
    b = _gpu_world(world, cam, k=16, packet_stack=1)
    np.testing.assert_array_equal(a["ids"], b["ids"])
    np.testing.assert_allclose(a["rgbT"], b["rgbT"], rtol=0, atol=1e-6)
    assert b["stats"]["fallbacks"] > 0
    world.close()


def test_world_update_moves_an_object(objects):
    gs, oscenes, gscenes = objects
    pl = _placements()
    world = R.World([(gscenes[i], M) for i, M in pl])
    moved = list(pl)
    moved[1] = (0, _affine(0.6 * _rot([0, 1, 0.3], -0.4), [-0.8, 0.9, 0.2]))
    moved = moved[:3]                                        # and one object removed
    world.update([(gscenes[i], M) for i, M in moved])
    cam = _cam()
    rays = O.camera_rays(cam)
    ref = O.world_render(oscenes, [i for i, _ in moved], [M for _, M in moved], rays, ids_cap=256)
    res = _gpu_world(world, cam, k=16)
    _check(res, ref, WorldResponder(oscenes, [i for i, _ in moved], [M for _, M in moved]), rays)
    world.close()


def test_world_rejects_bad_input(objects):
    gs, oscenes, gscenes = objects
    proxy = R.Scene.from_params(gs[1], form="proxy20")
    with pytest.raises(N.GrtxError, match="sphere-form"):
        R.World([(proxy, _affine(np.eye(3), [0, 0, 0]))])
    with pytest.raises(N.GrtxError, match="invertible"):
        R.World([(gscenes[0], _affine(np.diag([1.0, 0.0, 1.0]), [0, 0, 0]))])
    world = R.World([(gscenes[0], _affine(np.eye(3), [0, 0, 0]))])
    with pytest.raises(N.GrtxError, match="k = 8, 16 or 32"):
        R.render_world(world, _cam(), k=4)
    with pytest.raises(N.GrtxError, match="checkpoint or restart"):
        R.render_world(world, _cam(), traversal="single")
    world.close()
    proxy.close()
