"""Large incoherent scene with one mirror bounce and one glass ball (6M Gaussians over 100 m,
fisheye camera): mirror and refraction rays against the oracle's, the trace of primary and secondary rays on identical FP32
ray inputs against the FP64 oracle on sampled rays (k = 16 and 32), and the bounce composite.
Ray generation itself is checked against the oracle in test_gpu_parity.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2601_20429_gb300 import native as N  # noqa: E402
from paper_2601_20429_gb300 import render as R  # noqa: E402
from paper_2601_20429_gb300 import scenes  # noqa: E402
from tests.gpu_util import RGB_TOL, compare_hit_lists  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def outdoor():
    g, cam, mirror, cfg = scenes.config_outdoor()
    prim, sec, spix = O.mirror_rays(cam, mirror)
    S = O.Scene.from_params(g)
    sc = R.Scene.from_params(g)
    return g, cam, mirror, prim, sec, spix, S, sc


@pytest.fixture(scope="module")
def outdoor_both(outdoor):
    """Primary rays with one bounce off the mirror or through the glass ball, whichever is
    nearer (oracle)."""
    g, cam, mirror = outdoor[:3]
    glass = scenes.outdoor_glass()
    prim, sec, spix = O.secondary_rays(cam, [mirror], [glass])
    return glass, prim, sec, spix


def test_secondary_rays_match_oracle(outdoor, outdoor_both):
    g, cam, mirror = outdoor[:3]
    glass, prim, sec, spix = outdoor_both
    n = cam["width"] * cam["height"]
    dev = [torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"),
           torch.empty(n, device="cuda")]
    sdev = [torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"),
            torch.empty(n, device="cuda")]
    spd = torch.empty(n, dtype=torch.int32, device="cuda")
    ns = torch.zeros(1, dtype=torch.int32, device="cuda")
    N.grtx_secondary_rays(N.make_camera(cam), [N.make_mirror(mirror)], [N.make_glass(glass)], dev, sdev, spd, ns)
    torch.cuda.synchronize()
    m = int(ns.item())
    gp = spd[:m].cpu().numpy()
    assert len(spix) > 60000 and abs(m - len(spix)) <= max(2, len(spix) // 1000)
    both, gi, oi = np.intersect1d(gp, spix, return_indices=True)
    assert len(both) >= len(spix) - max(2, len(spix) // 1000)
    # rays through the ball away from its rim, where the entry point and the refraction are
    # well conditioned, match closely; rim rays (impact parameter above 0.98 R) more loosely
    c = np.asarray(glass["center"])
    hit = prim[0][both] + prim[3][both, None] * prim[1][both]
    on_ball = np.abs(np.linalg.norm(hit - c, axis=1) - glass["radius"]) < 1e-6
    u = prim[1][both] / np.linalg.norm(prim[1][both], axis=1, keepdims=True)
    b = np.linalg.norm(np.cross(c - prim[0][both], u), axis=1) / glass["radius"]
    assert on_ball.sum() > 5000
    keep = ~on_ball | (b < 0.98)
    tf = dev[3].cpu().numpy()
    np.testing.assert_allclose(tf[both][keep], prim[3][both][keep], rtol=2e-5)
    np.testing.assert_allclose(tf[both][~keep], prim[3][both][~keep], rtol=2e-4)
    assert np.isinf(tf[np.setdiff1d(np.arange(n), gp)]).mean() > 0.99
    so, sd = sdev[0][:m].cpu().numpy()[gi], sdev[1][:m].cpu().numpy()[gi]
    np.testing.assert_allclose(sd[keep], sec[1][oi][keep], atol=1e-4)
    np.testing.assert_allclose(so[keep], sec[0][oi][keep], atol=5e-4)
    stn = sdev[2][:m].cpu().numpy()[gi]
    np.testing.assert_array_equal(stn, np.float32(1e-3))


def test_glass_bounce_renders_like_the_oracle(outdoor, outdoor_both):
    """Trace the oracle's refracted and reflected secondary rays (as FP32) on the GPU and
    composite them: sampled pixels against the oracle's FP64 render and composite."""
    S, sc = outdoor[6], outdoor[7]
    glass, prim, sec, spix = outdoor_both
    p32, s32 = _f32(prim), _f32(sec)
    c = np.asarray(glass["center"])
    hit = prim[0][spix] + prim[3][spix, None] * prim[1][spix]
    through_glass = np.nonzero(np.abs(np.linalg.norm(hit - c, axis=1) - glass["radius"]) < 1e-6)[0]
    rng = np.random.default_rng(7)
    si = np.sort(rng.choice(through_glass, 64, replace=False))
    s_out = R.render(sc, None, rays=_to_dev(s32), k=16)
    p_out = R.render(sc, None, rays=_to_dev(p32), k=16)
    comb = p_out["rgbT"].clone()
    N.grtx_composite_bounce(comb, s_out["rgbT"], torch.from_numpy(spix).cuda(),
                            torch.tensor([len(spix)], dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    mp = spix[si]
    ref_p = S.render(tuple(a[mp].astype(np.float64) for a in p32))["out"]
    ref_s = S.render(tuple(a[si].astype(np.float64) for a in s32))["out"]
    got_s = s_out["rgbT"].cpu().numpy()[si].astype(np.float64)
    assert np.abs(got_s - ref_s).max() <= RGB_TOL
    assert (ref_s[:, 3] < 0.99).sum() > 10                       # the refracted rays see Gaussians
    ref_c = O.composite_bounce(ref_p, ref_s, np.arange(len(si), dtype=np.int32))
    assert np.abs(comb.cpu().numpy()[mp].astype(np.float64) - ref_c).max() <= 2 * RGB_TOL


def _f32(rays):
    return tuple(np.ascontiguousarray(a, dtype=np.float32) for a in rays)


def _to_dev(rays):
    return tuple(torch.from_numpy(a).cuda() for a in rays)


def test_mirror_rays_match_oracle(outdoor):
    g, cam, mirror, prim, sec, spix, S, sc = outdoor
    n = cam["width"] * cam["height"]
    dev = [torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"),
           torch.empty(n, device="cuda")]
    sdev = [torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"),
            torch.empty(n, device="cuda")]
    spd = torch.empty(n, dtype=torch.int32, device="cuda")
    ns = torch.zeros(1, dtype=torch.int32, device="cuda")
    N.grtx_mirror_rays(N.make_camera(cam), N.make_mirror(mirror), dev, sdev, spd, ns)
    torch.cuda.synchronize()
    m = int(ns.item())
    gp = spd[:m].cpu().numpy()
    assert abs(m - len(spix)) <= max(2, len(spix) // 2000)       # pixels on the rectangle's rim may differ
    assert len(spix) > 1000                                      # the mirror is in view
    both, gi, oi = np.intersect1d(gp, spix, return_indices=True)
    assert len(both) >= len(spix) - max(2, len(spix) // 2000)
    so = sdev[0][:m].cpu().numpy()[gi]
    sd = sdev[1][:m].cpu().numpy()[gi]
    np.testing.assert_allclose(so, sec[0][oi], atol=2e-5 * 20)
    np.testing.assert_allclose(sd, sec[1][oi], atol=2e-5)
    tf = dev[3].cpu().numpy()
    np.testing.assert_allclose(tf[both], prim[3][both], rtol=2e-5)
    assert np.isinf(tf[np.setdiff1d(np.arange(n), gp)]).mean() > 0.99


@pytest.mark.parametrize("k", [16, 32])
def test_outdoor_trace_and_bounce_on_identical_rays(outdoor, k):
    g, cam, mirror, prim, sec, spix, S, sc = outdoor
    p32, s32 = _f32(prim), _f32(sec)
    p_out = R.render(sc, None, rays=_to_dev(p32), k=k, ids_cap=256, want_n_blended=True)
    s_out = R.render(sc, None, rays=_to_dev(s32), k=k, ids_cap=256, want_n_blended=True)
    comb = p_out["rgbT"].clone()
    N.grtx_composite_bounce(comb, s_out["rgbT"], torch.from_numpy(spix).cuda(),
                            torch.tensor([len(spix)], dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    rng = np.random.default_rng(k)
    pi = np.sort(rng.choice(p32[0].shape[0], 96, replace=False))
    si = np.sort(rng.choice(len(spix), 64, replace=False))
    for rays, out, idx in ((p32, p_out, pi), (s32, s_out, si)):
        sub = tuple(a[idx].astype(np.float64) for a in rays)
        ref = S.render(sub, ids_cap=256)
        got = out["rgbT"].cpu().numpy()[idx].astype(np.float64)
        err = np.abs(got - ref["out"]).max(0)
        assert err.max() <= RGB_TOL, err
        gid, gnb = out["ids"].cpu().numpy()[idx], out["n_blended"].cpu().numpy()[idx]
        bad = compare_hit_lists(S, sub, gid, gnb, ref["ids"], ref["n_blend"])
        msgs = []
        for r in bad[:3]:
            a = [int(x) for x in gid[r, :gnb[r]]]
            b = [int(x) for x in ref["ids"][r, :ref["n_blend"][r]]]
            diff = sorted(set(a) ^ set(b))
            info = [(x, x in a, x in b) + S.response(x, sub[0][r], sub[1][r]) for x in diff[:6]]
            msgs.append(f"ray {r}: gpu {len(a)} ora {len(b)} first diff at "
                        f"{next((i for i, (u, v) in enumerate(zip(a, b)) if u != v), min(len(a), len(b)))}; "
                        f"(id, in gpu, in oracle, t, d2, alpha): {info}")
        assert not bad, "\n".join(msgs)
    # composite on the sampled mirror pixels: oracle primary + oracle secondary
    mp = spix[si]
    ref_p = S.render(tuple(a[mp].astype(np.float64) for a in p32))["out"]
    ref_s = S.render(tuple(a[si].astype(np.float64) for a in s32))["out"]
    ref_c = O.composite_bounce(ref_p, ref_s, np.arange(len(si), dtype=np.int32))
    got_c = comb.cpu().numpy()[mp].astype(np.float64)
    assert np.abs(got_c - ref_c).max() <= 2 * RGB_TOL
