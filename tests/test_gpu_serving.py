"""Serving (continuous batching over resident scenes): every request's image is the same
alone and in the mix (within the parity tolerance: the serving kernel inlines the same
trace code in another context, so FP contraction may differ by an ulp), requests admitted
while others run complete correctly, and the server's host-side errors are reported."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_20429_gb300 import native as N  # noqa: E402
from paper_2601_20429_gb300 import render as R  # noqa: E402
from paper_2601_20429_gb300 import scenes  # noqa: E402
from paper_2601_20429_gb300.serve import Server  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 2e-4


def _same(a, b):
    d = float((a - b).abs().max())
    assert d <= TOL, d
    return d


@pytest.fixture(scope="module")
def world():
    gs = [scenes.surface_scene(n=n, seed=40 + i) for i, n in enumerate((20_000, 50_000, 80_000))]
    sc = [R.Scene.from_params(g) for g in gs]
    reqs = scenes.request_stream(n_requests=24, n_scenes=3, seed=9,
                                 resolutions=((64, 64), (96, 80), (200, 120), (333, 217)))
    alone = []
    for r in reqs:
        out = R.render(sc[r["scene"]], r["camera"], k=16)["rgbT"]
        alone.append(out.clone())
    torch.cuda.synchronize()
    return sc, reqs, alone


def _bufs(reqs):
    return [torch.full((r["camera"]["width"] * r["camera"]["height"], 4), -1.0, device="cuda") for r in reqs]


def test_alone_equals_mix(world):
    sc, reqs, alone = world
    srv = Server(sc, k=16, max_rays_per_step=20_000, max_inflight=8)
    bufs = _bufs(reqs)
    done = srv.render_requests([(r["scene"], r["camera"], b, i) for i, (r, b) in enumerate(zip(reqs, bufs))])
    torch.cuda.synchronize()
    assert sorted(d["tag"] for d in done) == list(range(len(reqs)))
    assert all(d["status"] == 0 and d["t_done"] >= d["t_admit"] for d in done)
    worst = max(_same(a, b) for a, b in zip(alone, bufs))
    assert worst <= 1e-5
    srv.close()


def test_restart_traversal_serves_the_same_images(world):
    """The server with restart traversal (every round a warp packet) gives every request the
    image of a lone checkpointed render."""
    sc, reqs, alone = world
    srv = Server(sc, k=16, traversal="restart", max_rays_per_step=20_000, max_inflight=8)
    bufs = _bufs(reqs)
    done = srv.render_requests([(r["scene"], r["camera"], b, i) for i, (r, b) in enumerate(zip(reqs, bufs))])
    torch.cuda.synchronize()
    assert sorted(d["tag"] for d in done) == list(range(len(reqs)))
    worst = max(_same(a, b) for a, b in zip(alone, bufs))
    assert worst <= 1e-5
    srv.close()


def test_requests_admitted_while_others_run(world):
    sc, reqs, alone = world
    srv = Server(sc, k=16, max_rays_per_step=5_000, max_inflight=3)
    bufs = _bufs(reqs)
    first = [(r["scene"], r["camera"], b, i) for i, (r, b) in enumerate(zip(reqs[:12], bufs[:12]))]
    srv.submit(first)
    got = srv.poll(wait=True)
    inflight, pending = srv.load()
    assert inflight + pending + len(got) == 12
    srv.submit([(r["scene"], r["camera"], b, 12 + i) for i, (r, b) in enumerate(zip(reqs[12:], bufs[12:]))])
    while len(got) < len(reqs):
        got += srv.poll(wait=True)
    torch.cuda.synchronize()
    assert sorted(d["tag"] for d in got) == list(range(len(reqs)))
    for a, b in zip(alone, bufs):
        _same(a, b)
    # completions are reported in admission order within a step, never before admission
    assert all(d["t_done"] >= d["t_admit"] for d in got)
    srv.close()


def test_server_errors(world):
    sc, reqs, alone = world
    srv = Server(sc, k=16)
    buf = torch.empty((64 * 64, 4), device="cuda")
    with pytest.raises(N.GrtxError) as e:
        srv.submit([(7, reqs[0]["camera"], buf, 0)])
    assert e.value.status == 7            # GRTX_ERR_NOT_FOUND
    cam = dict(reqs[0]["camera"], width=0)
    with pytest.raises(N.GrtxError) as e:
        srv.submit([(0, cam, buf, 0)])
    assert e.value.status == 1
    assert srv.load() == (0, 0)
    srv.close()
    plain = R.Scene.from_params(scenes.surface_scene(n=1000, seed=1), form="proxy20")
    with pytest.raises(N.GrtxError):
        Server([plain], k=16)


@pytest.mark.slow
def test_serving_full_size_sampled_against_oracle():
    """The serving configuration at full size (four resident scenes of 0.5/1/2/3 M Gaussians)
    and requests from its Poisson stream, rendered through the server; sampled pixels of each
    request against the FP64 oracle on the same scene."""
    from oracle import oracle as O
    from tests.gpu_util import RGB_TOL, compare_hit_lists
    scs, reqs, cfg = scenes.config_serving(n_requests=40)
    gpu = [R.Scene.from_params(g) for g in scs]
    srv = Server(gpu, k=cfg["k"], max_rays_per_step=1 << 20, max_inflight=6)
    pick = [0, 1, 2, 3, 5, 8, 13, 21]
    bufs = [torch.empty((reqs[j]["camera"]["width"] * reqs[j]["camera"]["height"], 4), device="cuda") for j in pick]
    done = srv.render_requests([(reqs[j]["scene"], reqs[j]["camera"], b, j) for j, b in zip(pick, bufs)])
    torch.cuda.synchronize()
    assert sorted(d["tag"] for d in done) == sorted(pick)
    rng = np.random.default_rng(7)
    oracle_scenes = {}
    for j, b in zip(pick, bufs):
        sid = reqs[j]["scene"]
        if sid not in oracle_scenes:
            oracle_scenes[sid] = O.Scene.from_params(scs[sid])
        S = oracle_scenes[sid]
        cam = reqs[j]["camera"]
        rays = O.camera_rays(cam)
        idx = rng.choice(rays[0].shape[0], 12, replace=False)
        sub = tuple(a[idx] for a in rays)
        ref = S.render(sub, ids_cap=512)
        got = b.cpu().numpy()[idx].astype(np.float64)
        assert np.abs(got - ref["out"]).max() <= RGB_TOL
    srv.close()
