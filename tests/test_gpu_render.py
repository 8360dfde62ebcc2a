"""GPU parity of the per-frame path (R1-R4, brute force) against the oracle, through the C ABI.

Bit-exact: the projected splat parameters, the selected node set, the 64-bit fixed-point image
(for any tile size); the 8-bit tone-mapped image within +-1 LSB (depth and GPU paragraphs of
the paper; readings R-10..R-15)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

from gpu_helpers import to_dev, u8_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    return gblod


@pytest.fixture(scope="module")
def R(G):
    r = G.Renderer()
    yield r
    r.close()


def _cams():
    return {
        "outside": synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=320, height=200),
        "inside": synth.look_at((0.45, 0.55, 0.5), (0.9, 0.4, 0.6), width=333, height=197, z_near=1e-3),
        "grazing": synth.look_at((1.3, 0.5, 0.5), (0.5, 1.2, 0.4), width=160, height=120, vfov_deg=30.0),
    }


def test_projection_stage(G):
    rng = np.random.default_rng(3)
    n = 20000
    pts = np.concatenate([rng.uniform(-0.2, 1.2, (n, 3)), np.exp(rng.uniform(-4, 4, (n, 1)))], 1).astype(np.float32)
    h = np.exp(rng.uniform(-9, 0, n)).astype(np.float32)
    cam = _cams()["inside"]
    ahead = np.asarray(cam["eye"]) + 0.3 * np.asarray(cam["fwd"])  # certainly on screen
    pts[:4, :3] = ahead
    pts[:4, 3] = [np.nan, -1.0, 1e30, 0.0]
    for kernel in (0, 1):
        rp = G.make_params(kernel=kernel)
        got = G.project(*to_dev(pts, h), cam, rp).cpu().numpy()
        orp = O.rparams(kernel=kernel)
        want = np.array([O.project(cam, orp, *pts[i].tolist(), float(h[i])) for i in range(n)], np.int64)
        assert np.array_equal(got, want)
        assert (want[:, 0] == 1).sum() > 1000 and (want[:, 0] == -1).sum() >= 2


@pytest.mark.parametrize("view", ["outside", "inside", "grazing"])
@pytest.mark.parametrize("kernel", [0, 1])
def test_bruteforce_image(G, R, view, kernel):
    p = synth.tiny(30000, seed=21)
    cam = _cams()[view]
    img, acc = R.render_bruteforce(*to_dev(p.xyz, p.mass, p.h), cam, G.make_params(kernel=kernel))
    orp = O.rparams(kernel=kernel)
    want, st, nd = O.splat_particles(p.xyz, p.mass, p.h, cam, orp)
    assert R.status() == G.OK and st == 0
    got = G.u64(acc)
    assert np.array_equal(got, want)
    assert R.stats()["splats"] == nd
    assert u8_close(img.cpu().numpy(), O.tonemap(want, orp)) <= 1


@pytest.mark.parametrize("lam", [0.0, 8.0, None, float("inf")])
def test_lod_frame(G, R, lam):
    p = synth.tiny(60000, seed=22)
    n_max = 300
    t = G.build_lod(*to_dev(p.xyz, p.mass, p.h), n_max=n_max, seed=3)
    ot = O.build_tree(p.xyz, p.mass, p.h, seed=3, n_max=n_max)
    lam_v = G.default_lambda(n_max) if lam is None else lam
    for view, cam in _cams().items():
        img, acc = R.render(t, cam, G.make_params(lambda_px=lam_v))
        orp = O.rparams(lambda_px=lam_v)
        want, st, nd, npts = O.render_lod(ot, cam, orp)
        assert R.status() == G.OK and st == 0
        assert np.array_equal(R.last_selection(), O.select(ot, cam, orp)), view
        assert np.array_equal(G.u64(acc), want), view
        s = R.stats()
        assert s["splats"] == nd and s["points"] == npts
        assert u8_close(img.cpu().numpy(), O.tonemap(want, orp)) <= 1


def test_full_depth_lod_equals_bruteforce(G, R):
    p = synth.tiny(40000, seed=23)
    xyz = p.xyz.copy()
    xyz[:3] = [[1.2, 0.5, 0.5], [-0.3, 0.2, 0.1], [0.4, 0.4, -0.2]]
    d = to_dev(xyz, p.mass, p.h)
    t = G.build_lod(*d, n_max=150, seed=4)
    for cam in _cams().values():
        _, a = R.render(t, cam, G.make_params(lambda_px=0.0))
        _, b = R.render_bruteforce(*d, cam, G.make_params(lambda_px=0.0))
        assert torch.equal(a, b)


@pytest.mark.parametrize("tile", [(8, 8), (32, 8), (32, 16), (1, 1), (32, 32), (64, 16), (13, 7), (24, 32), (8, 64),
                                  (64, 8), (5, 50)])
def test_tiling_does_not_change_the_image(G, R, tile):
    p = synth.tiny(30000, seed=24)
    cam = _cams()["inside"]
    d = to_dev(p.xyz, p.mass, p.h)
    _, a = R.render_bruteforce(*d, cam, G.make_params())
    _, b = R.render_bruteforce(*d, cam, G.make_params(tile_w=tile[0], tile_h=tile[1]))
    assert torch.equal(a, b)


def test_counting_pixel_updates_keeps_the_image(G, R):
    p = synth.tiny(30000, seed=25)
    cam = _cams()["inside"]
    t = G.build_lod(*to_dev(p.xyz, p.mass, p.h), n_max=300, seed=2)
    _, a = R.render(t, cam, G.make_params())
    assert R.stats()["pixel_updates"] == 0
    _, b = R.render(t, cam, G.make_params(count_updates=True))
    n = R.stats()["pixel_updates"]
    assert torch.equal(a, b) and n > 0
    # the same frame counted by the tile shape that evaluates other pixel blocks gives the same count
    _, c = R.render(t, cam, G.make_params(count_updates=True, tile_w=16, tile_h=16))
    assert torch.equal(a, c) and R.stats()["pixel_updates"] == n
    # and the count is the oracle's for the points of the nodes it selects
    ot = O.build_tree(p.xyz, p.mass, p.h, seed=2, n_max=300)
    rp = O.rparams(lambda_px=G.default_lambda(300))
    sel = O.select(ot, cam, rp)
    idx = np.concatenate([np.arange(int(ot.nodes[i]["point_first"]), int(ot.nodes[i]["point_first"])
                                    + int(ot.nodes[i]["point_count"])) for i in sel])
    assert n == O.count_updates(ot.pts4[idx], ot.hs[idx], cam, rp)


@pytest.mark.parametrize("parts", [3, 17, 150])
def test_split_frames_give_the_same_image(G, R, parts):
    """A frame whose records exceed the budget is binned in several passes: same image."""
    p = synth.tiny(60000, seed=26)
    d = to_dev(p.xyz, p.mass, p.h)
    t = G.build_lod(*d, n_max=300, seed=3)
    for cam in _cams().values():
        _, a = R.render_bruteforce(*d, cam, G.make_params())
        pairs = R.stats()["pairs"]
        budget = max(1, pairs // parts)
        _, b = R.render_bruteforce(*d, cam, G.make_params(record_budget=budget))
        assert R.stats()["pairs"] == pairs
        assert torch.equal(a, b)
        _, c = R.render(t, cam, G.make_params(lambda_px=10.0))
        s1 = R.stats()
        _, e = R.render(t, cam, G.make_params(lambda_px=10.0, record_budget=budget))
        s2 = R.stats()
        assert torch.equal(c, e)
        assert all(s1[k] == s2[k] for k in s1 if k != "pixel_updates_total")


def test_fixed_tone_range(G, R):
    p = synth.tiny(30000, seed=25)
    cam = _cams()["outside"]
    lo, hi = 1e-3, 50.0
    img, acc = R.render_bruteforce(*to_dev(p.xyz, p.mass, p.h), cam,
                                   G.make_params(tone_auto=False, tone_lo=lo, tone_hi=hi))
    want = O.tonemap(G.u64(acc), O.rparams(tone_auto=0, tone_lo=lo, tone_hi=hi))
    assert u8_close(img.cpu().numpy(), want) <= 1


def test_edge_cases(G, R):
    cam = _cams()["outside"]
    e = np.zeros((0, 3), np.float32)
    z = np.zeros(0, np.float32)
    img, acc = R.render_bruteforce(*to_dev(e, z, z), cam)
    assert not acc.any() and not img.any()
    t = G.build_lod(*to_dev(e, z, z), n_max=4)
    img, acc = R.render(t, cam)
    assert not acc.any()
    # everything behind the camera or outside the view
    p = synth.uniform(1000, seed=3)
    xyz = p.xyz.copy()
    xyz[:, 2] -= 5.0
    img, acc = R.render_bruteforce(*to_dev(xyz, p.mass, p.h), cam)
    assert not acc.any() and R.stats()["splats"] == 0
    # one particle on a pixel centre, tiny image, splats straddling the border
    cam1 = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=3, height=2)
    q = np.array([[0.5, 0.5, 0.5], [0.2, 0.8, 0.4], [0.9, 0.1, 0.3]], np.float32)
    img, acc = R.render_bruteforce(*to_dev(q, np.ones(3, np.float32), np.full(3, 0.05, np.float32)), cam1)
    want, _, _ = O.splat_particles(q, np.ones(3, np.float32), np.full(3, 0.05, np.float32), cam1, O.rparams())
    assert np.array_equal(G.u64(acc), want)


def test_amplitude_range_is_reported(G, R):
    cam = _cams()["outside"]
    q = np.array([[0.5, 0.5, 0.5], [0.4, 0.5, 0.5]], np.float32)
    h = np.array([1e-6, 1e-6], np.float32)  # sigma clamps to 0.5 px
    w = np.array([1e9, 1.0], np.float32)    # amplitude beyond 2^48 for the first
    _, acc = R.render_bruteforce(*to_dev(q, w, h), cam)
    assert R.status(reset=True) == G.ERR_RANGE
    assert R.status() == G.OK
    want, st, _ = O.splat_particles(q, w, h, cam, O.rparams())
    assert st == O.ERR_RANGE and np.array_equal(G.u64(acc), want)


def test_invalid_arguments(G, R):
    cam = dict(_cams()["outside"], width=0)
    p = synth.uniform(10, seed=1)
    with pytest.raises(G.GblodError) as e:
        R.render_bruteforce(*to_dev(p.xyz, p.mass, p.h), cam)
    assert e.value.code == G.ERR_INVALID_ARG
    with pytest.raises(G.GblodError):
        R.render_bruteforce(*to_dev(p.xyz, p.mass, p.h), _cams()["outside"], G.make_params(tile_w=65))
    with pytest.raises(G.GblodError):
        R.render_bruteforce(*to_dev(p.xyz, p.mass, p.h), _cams()["outside"], G.make_params(tile_w=64, tile_h=64))
    with pytest.raises(G.GblodError):
        R.render_bruteforce(*to_dev(p.xyz, p.mass, p.h), _cams()["outside"], G.make_params(tile_w=17, tile_h=60))
    with pytest.raises(G.GblodError):  # 5 columns of strips x 2 rows: more than 8 warps
        R.render_bruteforce(*to_dev(p.xyz, p.mass, p.h), _cams()["outside"], G.make_params(tile_w=40, tile_h=24))
    with pytest.raises(G.GblodError):
        R.render_bruteforce(*to_dev(p.xyz, p.mass, p.h), _cams()["outside"], G.make_params(sigma_min_px=0.0))


def test_mid_workload_full_size_frames(G, R):
    """Full 2^24-particle mid workload, 1920x1080, frames of the benchmark's fly-through."""
    p = synth.mid()
    d = to_dev(p.xyz, p.mass, p.h)
    t = G.build_lod(*d, n_max=16000, seed=1)
    ot = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=16000)
    lam = G.default_lambda(16000)
    for k in (0, 239):
        cam = synth.helix_view(k)
        img, acc = R.render(t, cam, G.make_params(lambda_px=lam))
        orp = O.rparams(lambda_px=lam)
        want, st, nd, npts = O.render_lod(ot, cam, orp)
        assert np.array_equal(R.last_selection(), O.select(ot, cam, orp))
        assert np.array_equal(G.u64(acc), want)
        assert u8_close(img.cpu().numpy(), O.tonemap(want, orp)) <= 1
    cam = synth.helix_view(120)
    _, acc = R.render_bruteforce(*d, cam, G.make_params())
    want, _, _ = O.splat_particles(p.xyz, p.mass, p.h, cam, O.rparams())
    assert np.array_equal(G.u64(acc), want)


def _at_pixel(cam, u, v, d):
    """World point at depth d along the view whose projection is pixel position (u, v)."""
    e, r, up, f = (np.asarray(cam[k], np.float64) for k in ("eye", "right", "up", "fwd"))
    return e + d * f + ((u - cam["cx"]) * d / cam["f_px"]) * r - ((v - cam["cy"]) * d / cam["f_px"]) * up


def _box_sides(cam, rp, pts4, h):
    """Coverage only: how many drawn points have a clipped pixel box of at most 8 x 8 pixels (the
    library's rule, restated: support bound sqrt(2^47 / S) + 2 in 1/256 px around the centre)."""
    small = binned = 0
    for i in range(len(h)):
        r = O.project(cam, rp, *pts4[i].tolist(), float(h[i]))
        if r[0] != 1:
            continue
        U, V, S = r[1], r[2], r[3]
        rr = int(np.sqrt(np.float32(2.0 ** 47) / np.float32(S))) + 2
        x0, x1 = max(-((rr + 128 - U) >> 8), 0), min((U - 128 + rr) >> 8, cam["width"] - 1)
        y0, y1 = max(-((rr + 128 - V) >> 8), 0), min((V - 128 + rr) >> 8, cam["height"] - 1)
        if x0 > x1 or y0 > y1:
            continue
        if x1 - x0 < 8 and y1 - y0 < 8:
            small += 1
        else:
            binned += 1
    return small, binned


def test_small_boxes_splatted_without_binning(G, R):
    """Points whose pixel box is at most 8 x 8 skip the tile records and are added to the image by
    the scatter pass: sigma from the 0.5 px clamp to 3 px (boxes on both sides of the rule), image
    borders and corners, 400 coincident points (same-pixel atomics) and large splats centred off
    screen that reach only a corner's few pixels.  Same image and pixel-update count as the oracle,
    for two tile shapes, brute force and full-depth LOD."""
    cam = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=96, height=64)
    rng = np.random.default_rng(31)
    d = 1.5
    n = 6000
    u = rng.uniform(-4.0, cam["width"] + 4.0, n)
    v = rng.uniform(-4.0, cam["height"] + 4.0, n)
    sigma = np.exp(rng.uniform(np.log(0.3), np.log(3.0), n))
    xyz = np.array([_at_pixel(cam, a, b, d) for a, b in zip(u, v)])
    h = sigma * d / cam["f_px"]
    # coincident points on one pixel, all with the clamped sigma
    xyz[:400] = _at_pixel(cam, 40.3, 21.7, d)
    h[:400] = 1e-5
    # large splats (sigma 6 px) whose support reaches only a few pixels of a corner
    for i, (cu, cv) in enumerate([(-3.2, -2.9), (cam["width"] + 3.3, -3.1), (-2.8, cam["height"] + 3.4),
                                  (cam["width"] + 3.1, cam["height"] + 2.7), (-4.0, 30.0)]):
        xyz[400 + i] = _at_pixel(cam, cu, cv, d)
        h[400 + i] = 2.0 * d / cam["f_px"]
    xyz = xyz.astype(np.float32)
    h = h.astype(np.float32)
    mass = rng.uniform(0.5, 2.0, n).astype(np.float32)
    dv = to_dev(xyz, mass, h)
    rp = O.rparams()
    want, st, nd = O.splat_particles(xyz, mass, h, cam, rp)
    assert st == 0 and nd > 5000
    pts4 = np.concatenate([xyz, mass[:, None]], 1).astype(np.float32)
    n_upd = O.count_updates(pts4, h, cam, rp)
    small, binned = _box_sides(cam, rp, pts4, h)
    assert small > 3000 and binned > 1500  # both sides of the rule are exercised
    for tile in ((64, 16), (8, 8)):
        _, acc = R.render_bruteforce(*dv, cam, G.make_params(tile_w=tile[0], tile_h=tile[1], count_updates=True))
        assert R.status() == G.OK
        assert np.array_equal(G.u64(acc), want), tile
        s = R.stats()
        assert s["splats"] == nd and s["pixel_updates"] == n_upd, tile
    # full depth equals brute force while no depth-21 node is lossy: the 400 coincident points share
    # one depth-21 cell, so n_max must exceed 400
    t = G.build_lod(*dv, n_max=1000, seed=5)
    assert not np.any(t.export()["nodes"]["flags"] & G.NODE_LOSSY)
    _, a = R.render(t, cam, G.make_params(lambda_px=0.0, count_updates=True))
    assert np.array_equal(G.u64(a), want) and R.stats()["pixel_updates"] == n_upd
    t.free()
