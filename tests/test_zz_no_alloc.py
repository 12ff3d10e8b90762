"""The allocation-free forward trace (grtx_trace_forward_noalloc) gives the image of the
regular entry point. It exists for callers that may not allocate device memory while they
render; it keeps its scratch in a fixed library-owned array instead. Collected last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_20429_gb300 import native as N  # noqa: E402
from paper_2601_20429_gb300 import render as R  # noqa: E402
from paper_2601_20429_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 2e-4


@pytest.mark.parametrize("form,k", [("sphere", 16), ("sphere", 4), ("proxy20", 8)])
def test_noalloc_matches_regular_entry_point_twice(form, k):
    g = scenes.surface_scene(n=60_000, seed=21)
    cam = scenes.pinhole_camera(320, 200, (0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 60.0)
    sc = R.Scene.from_params(g, form=form)
    ref = R.render(sc, cam, k=k)["rgbT"]
    p = R.trace_params(k=k, alpha_min=sc.alpha_min)
    c = N.make_camera(cam)
    for _ in range(2):                      # two calls in a row share the fixed scratch
        out = torch.full_like(ref, -1.0)
        N.grtx_trace_forward_noalloc(sc.handle, c, p, out)
        torch.cuda.synchronize()
        assert float((out - ref).abs().max()) <= TOL
    assert float(ref[:, 3].min()) < 0.5      # the frame actually hits Gaussians
    sc.close()


@pytest.mark.parametrize("traversal", ["checkpoint", "restart"])
def test_noalloc_on_a_fresh_scene_allocates_nothing(traversal):
    """On a scene that no regular trace has touched, the allocation-free trace leaves the
    scene's own workspace unallocated and the device's free memory unchanged across a call
    (the first call on a device may still load the library's device code, so it comes
    first), and gives the regular entry point's image in both traversal modes."""
    g = scenes.surface_scene(n=60_000, seed=22)
    cam = scenes.pinhole_camera(256, 160, (0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 60.0)
    sc = R.Scene.from_params(g)
    p = R.trace_params(k=16, traversal=traversal, alpha_min=sc.alpha_min)
    c = N.make_camera(cam)
    n = cam["width"] * cam["height"]
    outs = [torch.full((n, 4), -1.0, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    N.grtx_trace_forward_noalloc(sc.handle, c, p, outs[0])
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    N.grtx_trace_forward_noalloc(sc.handle, c, p, outs[1])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert sc.info()["bytes_workspace"] == 0
    ref = R.render(sc, cam, k=16, traversal=traversal)["rgbT"]
    torch.cuda.synchronize()
    for out in outs:
        assert float((out - ref).abs().max()) <= TOL
    assert float(ref[:, 3].min()) < 0.5
    sc.close()


def test_noalloc_rejects_capacities_beyond_its_scratch():
    g = scenes.tiny_scene(seed=0, n=500)
    cam = scenes.pinhole_camera(16, 16, (0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 60.0)
    sc = R.Scene.from_params(g)
    p = R.trace_params(k=8, alpha_min=sc.alpha_min, ckpt_capacity=65536, evict_capacity=65536)
    out = torch.empty((256, 4), device="cuda")
    with pytest.raises(N.GrtxError) as e:
        N.grtx_trace_forward_noalloc(sc.handle, N.make_camera(cam), p, out)
    assert e.value.status == 1 and "scratch" in str(e.value)
    sc.close()
