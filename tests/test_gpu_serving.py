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


def test_small_request_completes_before_the_large_one_in_its_step(world):
    """A request is reported when its own tiles are done, not when its whole step is: in one
    step holding a 3840x2160 view (about 50 times as many 32-ray tiles as the launch has warps)
    and a 64x64 view from the same pose, submitted in that order, the small view's tiles are
    handed out first and it completes before the large one, with both images equal to the lone
    renders. (A request's latency is at least its slowest tile's, up to a millisecond or two
    for rays through dense Gaussians, so the large view must take several times that.)"""
    sc, reqs, alone = world
    big_cam = scenes.pinhole_camera(3840, 2160, (0.0, 0.5, -3.0), (0.0, 0.0, 0.0), 60.0)
    small_cam = scenes.pinhole_camera(64, 64, (0.0, 0.5, -3.0), (0.0, 0.0, 0.0), 60.0)
    big_alone = R.render(sc[2], big_cam, k=16)["rgbT"].clone()
    small_alone = R.render(sc[2], small_cam, k=16)["rgbT"].clone()
    srv = Server(sc, k=16, max_rays_per_step=1 << 24, max_inflight=8)
    big_buf = torch.full_like(big_alone, -1.0)
    small_buf = torch.full_like(small_alone, -1.0)
    for _ in range(3):
        srv.submit([(2, big_cam, big_buf, 0), (2, small_cam, small_buf, 1)])
        got = []
        while len(got) < 2:
            got += srv.poll(wait=True)
        torch.cuda.synchronize()
        done = {c["tag"]: c for c in got}
        assert done[1]["t_done"] < done[0]["t_done"]
    _same(big_alone, big_buf)
    _same(small_alone, small_buf)
    srv.close()


def test_new_requests_join_the_running_launch(world):
    """Requests submitted while a step launch still runs are appended to that launch instead of
    starting another, and render the lone images."""
    sc, reqs, alone = world
    big_cam = scenes.pinhole_camera(1920, 1080, (0.0, 0.5, -3.0), (0.0, 0.0, 0.0), 60.0)
    big_alone = R.render(sc[2], big_cam, k=16)["rgbT"].clone()
    srv = Server(sc, k=16, max_inflight=16)
    bufs = _bufs(reqs)
    big_buf = torch.full_like(big_alone, -1.0)
    srv.submit([(2, big_cam, big_buf, 100)])
    got = srv.poll()                               # starts the launch over the large view
    # the launch is still tracing the large view (about a millisecond of work)
    srv.submit([(r["scene"], r["camera"], b, i) for i, (r, b) in enumerate(zip(reqs[:5], bufs[:5]))])
    while len(got) < 6:
        got += srv.poll(wait=True)
    torch.cuda.synchronize()
    info = srv.info()
    assert info["n_launches"] == 1 and info["n_appends"] >= 1, info
    assert sorted(d["tag"] for d in got) == [0, 1, 2, 3, 4, 100]
    _same(big_alone, big_buf)
    for j in range(5):
        _same(alone[j], bufs[j])
    srv.close()


@pytest.mark.parametrize("linger_us,guard", [(0, True), (3, True), (30, True), (0, False), (3, False)])
def test_short_waits_lose_no_tiles(world, linger_us, guard):
    """With waits too short to bridge the gaps between submissions, launches end while work is
    appended to them (without the host's guard, often: it then appends to any launch it has
    not seen stop): tiles a warp gave up on, and items published after the last warp stopped,
    are traced by later launches, and every image is still the lone render."""
    sc, reqs, alone = world
    srv = Server(sc, k=16, max_rays_per_step=6_000, max_inflight=6, linger_us=linger_us, append_guard=guard)
    bufs = _bufs(reqs)
    got = []
    for i, (r, b) in enumerate(zip(reqs, bufs)):
        srv.submit([(r["scene"], r["camera"], b, i)])
        got += srv.poll()
    while len(got) < len(reqs):
        got += srv.poll(wait=True)
    torch.cuda.synchronize()
    assert sorted(d["tag"] for d in got) == list(range(len(reqs)))
    worst = max(_same(a, b) for a, b in zip(alone, bufs))
    assert worst <= 1e-5
    info = srv.info()
    print(f"linger {linger_us} us, guard {guard}: {info['n_launches']} launches, {info['n_appends']} appends, "
          f"{info['n_retried_tiles']} tiles retried")
    srv.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_schedules_give_the_lone_images(world, seed):
    """Randomised use of the server: requests submitted in random bursts between blocking and
    non-blocking polls, under a random wait of idle warps (0, 5 us, the default, 200 ms), a
    random publication order (admission order, the default deadline weight, smallest first),
    small or default publications, and a segment table of 4 x 2 pieces (launches close when
    it fills). Every request completes once, with the lone image."""
    sc, reqs, alone = world
    rng = np.random.default_rng(seed)
    linger = [0.0, 5.0, None, 200_000.0][rng.integers(4)]
    order = [0.0, None, 1e6][rng.integers(3)]
    chunk = int(rng.choice([0, 4096, 20_000]))
    srv = Server(sc, k=16, max_rays_per_step=chunk, max_inflight=2, linger_us=linger, size_ns_per_ray=order)
    bufs = _bufs(reqs)
    todo = list(rng.permutation(len(reqs)))
    got = []
    while todo or len(got) < len(reqs):
        if todo and rng.random() < 0.5:
            burst = [int(todo.pop()) for _ in range(min(len(todo), int(rng.integers(1, 5))))]
            srv.submit([(reqs[j]["scene"], reqs[j]["camera"], bufs[j], j) for j in burst])
        got += srv.poll(wait=bool(rng.random() < 0.3) and not todo)
    torch.cuda.synchronize()
    assert sorted(d["tag"] for d in got) == list(range(len(reqs)))
    assert all(d["status"] == 0 and d["t_done"] >= d["t_admit"] for d in got)
    for a, b in zip(alone, bufs):
        _same(a, b)
    info = srv.info()
    print(f"seed {seed}: linger {linger}, order {order}, chunk {chunk}: {info['n_launches']} launches, "
          f"{info['n_appends']} appends, {info['n_retried_tiles']} tiles retried")
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
    for bad in (-1, 2_000_000):
        with pytest.raises(N.GrtxError) as e:
            N.check(N.lib().grtx_server_set_linger(srv.handle, int(bad * 1000)), "grtx_server_set_linger")
        assert e.value.status == 1
    srv.close()
    plain = R.Scene.from_params(scenes.surface_scene(n=1000, seed=1), form="proxy20")
    with pytest.raises(N.GrtxError):
        Server([plain], k=16)


# Small list capacities for the budget tests: one 128-ray block of lists is then
# 128 * (2 * 16 + 32) * 8 = 64 KiB, the size of one 64x64 output (capacity overflows fall back
# to exact restarts, so the images do not change).
CAPS = dict(ckpt_capacity=16, evict_capacity=32)
PER_BLOCK = 128 * (2 * 16 + 32) * 8
OUT64 = 64 * 64 * 16


def _budget_for(n_outputs):
    """A budget of one block of lists (its half for lists holds one block, not two) and an
    output arena of n 64x64 outputs plus less than one more (the queue counters and the
    segment tables of 8 requests take under 16 KiB)."""
    return PER_BLOCK + n_outputs * OUT64 + 16384


def test_memory_budget_holds_requests_until_outputs_are_released(world):
    """Under a budget whose output arena holds one 64x64 image, server-owned requests are
    admitted one at a time: the others stay pending while an output is held, and the next is
    admitted only after release. Every image equals the lone render; the server's device
    memory never exceeds the budget."""
    sc, reqs, alone = world
    budget = _budget_for(1)
    srv = Server(sc, k=16, mem_budget_bytes=budget, max_inflight=8, **CAPS)
    inf = srv.info()
    assert inf["device_bytes"] <= budget and inf["n_step_slots"] == 1 and inf["blocks_per_step"] == 1
    assert inf["list_bytes"] == PER_BLOCK
    assert OUT64 <= inf["arena_bytes"] < 2 * OUT64
    small = [j for j, r in enumerate(reqs) if (r["camera"]["width"], r["camera"]["height"]) == (64, 64)][:4]
    assert len(small) >= 3
    srv.submit([(reqs[j]["scene"], reqs[j]["camera"], None, j) for j in small])
    seen = []
    while len(seen) < len(small):
        got = srv.poll(wait=True)
        inf = srv.info()
        assert inf["arena_used"] <= inf["arena_bytes"] and inf["n_inflight"] <= 1
        for c in got:
            assert c["status"] == 0 and c["d_rgbT"]
            torch.cuda.synchronize()
            # held: nothing else is admitted while this output is not released
            assert srv.poll() == []
            i2 = srv.info()
            assert i2["n_inflight"] == 0 and i2["n_pending"] == len(small) - len(seen) - 1
            _same(alone[c["tag"]], c["rgbT"])
            seen.append(c["tag"])
            srv.release(c)
    assert sorted(seen) == sorted(small)
    assert srv.info()["arena_used"] == 0
    srv.close()


def test_memory_budget_mixes_owned_and_caller_outputs_and_rejects_oversize(world):
    """Under a budget whose arena holds two 64x64 outputs: a request larger than the arena is
    rejected at submission with GRTX_ERR_OOM (nothing queued); requests that bring their own
    buffer need no arena; owned and caller outputs mixed all give the lone images. Without a
    budget a server-owned output is an argument error; a budget below one block of lists is
    rejected at creation."""
    sc, reqs, alone = world
    srv = Server(sc, k=16, mem_budget_bytes=_budget_for(2), max_inflight=8, **CAPS)
    assert 2 * OUT64 <= srv.info()["arena_bytes"] < 3 * OUT64
    big = next(r for r in reqs if r["camera"]["width"] * r["camera"]["height"] > 3 * 64 * 64)
    with pytest.raises(N.GrtxError) as e:
        srv.submit([(big["scene"], big["camera"], None, 99)])
    assert e.value.status == 2                    # GRTX_ERR_OOM
    assert srv.load() == (0, 0)
    bufs = _bufs(reqs)
    small = {j for j, r in enumerate(reqs) if (r["camera"]["width"], r["camera"]["height"]) == (64, 64)}
    batch = [(r["scene"], r["camera"], None if j in small else bufs[j], j) for j, r in enumerate(reqs)]
    srv.submit(batch)
    done = 0
    while done < len(reqs):
        for c in srv.poll(wait=True):
            assert c["status"] == 0
            j = c["tag"]
            torch.cuda.synchronize()
            _same(alone[j], c["rgbT"] if j in small else bufs[j])
            if j in small:
                srv.release(c)
            done += 1
    with pytest.raises(N.GrtxError):
        srv.release(12345)                        # not a live server-owned output
    srv.close()
    plain = Server(sc, k=16)
    with pytest.raises(N.GrtxError) as e:
        plain.submit([(0, reqs[0]["camera"], None, 0)])
    assert e.value.status == 1
    assert plain.info()["n_step_slots"] == 2 and plain.info()["arena_bytes"] == 0
    plain.close()
    with pytest.raises(N.GrtxError) as e:
        Server(sc, k=16, mem_budget_bytes=PER_BLOCK, max_inflight=8, **CAPS)   # half is below a block
    assert e.value.status == 1
    big_budget = Server(sc, k=16, mem_budget_bytes=16 << 30)                  # lists of full step slots
    inf = big_budget.info()
    assert inf["n_step_slots"] >= 2 and inf["device_bytes"] <= 16 << 30 and inf["arena_bytes"] >= (8 << 30) - (1 << 20)
    big_budget.close()


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
