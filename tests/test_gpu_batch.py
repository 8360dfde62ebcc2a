"""Batched multi-view rendering (NEXT-1 of the hot path): views with different cameras,
resolutions and octrees rendered by one set of launches without host waits.  Each view of a batch
must equal the same view rendered alone, bit for bit; a CUDA-graph replay must equal the direct
call; a batch beyond its reserved capacity must be flagged."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    return gblod


@pytest.fixture(scope="module")
def scene(G):
    a = synth.tiny(40000, seed=41)
    b = synth.clustered(60000, 48, 0.1, 0.25, seed=42)
    ta = G.build_lod(*to_dev(a.xyz, a.mass, a.h), n_max=400, seed=5)
    tb = G.build_lod(*to_dev(b.xyz, b.mass, b.h), n_max=300, seed=6)
    cams = [synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=320, height=200),
            synth.look_at((0.45, 0.55, 0.5), (0.9, 0.4, 0.6), width=257, height=131, z_near=1e-3),
            synth.look_at((1.3, 0.5, 0.5), (0.5, 1.2, 0.4), width=160, height=120, vfov_deg=30.0),
            synth.look_at((0.2, 0.9, 0.1), (0.5, 0.5, 0.5), width=96, height=300),
            synth.look_at((0.5, -0.4, 0.5), (0.5, 0.5, 0.5), width=640, height=360)]
    return (a, ta), (b, tb), cams


def _views(dev, pairs):
    out = []
    for tree, cam in pairs:
        img = torch.full((cam["height"], cam["width"]), 3, dtype=torch.uint8, device=dev)
        acc = torch.full((cam["height"], cam["width"]), 77, dtype=torch.int64, device=dev)
        out.append((tree, cam, img, acc))
    return out


def test_batch_equals_views_alone(G, scene):
    (_, ta), (_, tb), cams = scene
    dev = torch.device("cuda", 0)
    pairs = [(ta, cams[0]), (tb, cams[1]), (ta, cams[2]), (tb, cams[3]), (tb, cams[4]), (ta, cams[1])]
    views = _views(dev, pairs)
    r = G.Renderer()
    for lam in (None, 0.0, 30.0):
        par = G.make_params(lambda_px=lam)
        r.reserve_batch(views, par, record_capacity=1 << 22)
        r.render_batch(views, par)
        torch.cuda.synchronize()
        assert r.status() == G.OK
        alone = G.Renderer()
        for tree, cam, img, acc in views:
            im1, ac1 = alone.render(tree, cam, par)
            assert torch.equal(acc, ac1)
            assert torch.equal(img, im1)
        alone.close()
    r.close()


def test_batch_matches_the_oracle(G, scene):
    (a, ta), _, cams = scene
    dev = torch.device("cuda", 0)
    views = _views(dev, [(ta, cams[0]), (ta, cams[2])])
    r = G.Renderer()
    par = G.make_params(lambda_px=20.0)
    r.reserve_batch(views, par)
    r.render_batch(views, par)
    torch.cuda.synchronize()
    ot = O.build_tree(a.xyz, a.mass, a.h, seed=5, n_max=400)
    for _, cam, img, acc in views:
        want, st, _, _ = O.render_lod(ot, cam, O.rparams(lambda_px=20.0))
        assert np.array_equal(G.u64(acc), want)
    r.close()


def test_graph_replay_equals_direct_call(G, scene):
    (_, ta), (_, tb), cams = scene
    dev = torch.device("cuda", 0)
    views = _views(dev, [(ta, cams[0]), (tb, cams[4]), (tb, cams[1])])
    r = G.Renderer()
    par = G.make_params()
    r.reserve_batch(views, par, record_capacity=1 << 22)
    r.render_batch(views, par)
    torch.cuda.synchronize()
    want = [acc.clone() for _, _, _, acc in views]
    want_img = [img.clone() for _, _, img, _ in views]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        r.render_batch(views, par)  # warm up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            r.render_batch(views, par, stream=s)
    torch.cuda.synchronize()
    for _, _, img, acc in views:
        acc.fill_(5)
        img.fill_(9)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for (_, _, img, acc), w, wi in zip(views, want, want_img):
            assert torch.equal(acc, w) and torch.equal(img, wi)
    assert r.status() == G.OK
    r.close()


def test_capacity_overflow_is_flagged(G, scene):
    (_, ta), _, cams = scene
    dev = torch.device("cuda", 0)
    views = _views(dev, [(ta, cams[0]), (ta, cams[4])])
    r = G.Renderer()
    par = G.make_params()
    r.reserve_batch(views, par, record_capacity=100)
    r.render_batch(views, par)
    torch.cuda.synchronize()
    assert r.status(reset=True) == G.ERR_CAPACITY
    r.reserve_batch(views, par, record_capacity=1 << 22)
    r.render_batch(views, par)
    assert r.status() == G.OK
    r.close()


def test_unreserved_batch_is_rejected(G, scene):
    (_, ta), _, cams = scene
    dev = torch.device("cuda", 0)
    r = G.Renderer()
    with pytest.raises(G.GblodError) as e:
        r.render_batch(_views(dev, [(ta, cams[0])]))
    assert e.value.code == G.ERR_INVALID_ARG
    r.close()


def test_autotuner_picks_a_tile_and_keeps_the_image(G, scene):
    (_, ta), (_, tb), cams = scene
    dev = torch.device("cuda", 0)
    views = _views(dev, [(ta, cams[0]), (tb, cams[4])])
    r = G.Renderer()
    G.Renderer.autotune_cache_clear()
    l0 = G.launch_count()
    par, ms = r.autotune(views, G.make_params(), record_capacity=1 << 22)
    l1 = G.launch_count()
    assert (par.tile_w, par.tile_h) in [(16, 16), (32, 16), (16, 32), (32, 32), (64, 16)] and ms > 0
    # the same batch again: served from the cache with a single measuring render
    par2, ms2 = r.autotune(views, G.make_params(), record_capacity=1 << 22)
    l2 = G.launch_count()
    assert (par2.tile_w, par2.tile_h) == (par.tile_w, par.tile_h) and ms2 == ms
    assert (l2 - l1) * 10 < (l1 - l0)
    r.render_batch(views, par)
    torch.cuda.synchronize()
    alone = G.Renderer()
    for tree, cam, _, acc in views:
        _, ac1 = alone.render(tree, cam, G.make_params())
        assert torch.equal(acc, ac1)
    alone.close()
    r.close()


def test_batch_with_off_image_blobs_and_pixel_piles_matches_the_oracle(G):
    # Full-depth frames (every leaf particle drawn) of two views of one octree, batched, against the
    # oracle: points far below a pixel (the small-box walk of the batched projection, pairs tagged
    # with their view), 2,000 points on one spot, and large blobs centred off each image whose
    # visible sliver or clipped corner box is small (64-bit distances in the walk).
    rng = np.random.default_rng(91)
    n = 40000
    xyz = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    h = np.full(n, 3e-4, np.float32)
    h[: n // 10] = rng.uniform(0.002, 0.02, n // 10).astype(np.float32)
    xyz[n // 10: n // 10 + 2000] = (0.5, 0.5, 0.5)
    mass = np.ones(n, np.float32)
    cams = [synth.look_at((0.5, 0.5, -1.2), (0.5, 0.5, 0.5), width=640, height=360),
            synth.look_at((0.5, 0.5, -1.2), (0.5, 0.5, 0.5), width=333, height=197)]
    D = 1.7
    for j, cam in enumerate(cams):
        W, H, F = cam["width"], cam["height"], cam["f_px"]
        for k, (u, v, sig) in enumerate([(-296.0, 100.0, 100.0), (W + 296.0, 50.0, 100.0), (-294.0, -294.0, 100.0),
                                         (W + 294.0, H + 294.0, 100.0), (100.0, -116.0, 40.0)]):
            xyz[500 + 10 * j + k] = (0.5 - (u - cam["cx"]) * D / F, 0.5 - (v - cam["cy"]) * D / F, 0.5)
            h[500 + 10 * j + k] = sig * D / F
    t = G.build_lod(*to_dev(xyz, mass, h), n_max=500, seed=4)
    dev = torch.device("cuda", 0)
    views = _views(dev, [(t, cams[0]), (t, cams[1])])
    r = G.Renderer()
    par = G.make_params(lambda_px=0.0)
    r.reserve_batch(views, par, record_capacity=1 << 22)
    r.render_batch(views, par)
    torch.cuda.synchronize()
    assert r.status() == G.OK
    ot = O.build_tree(xyz, mass, h, seed=4, n_max=500)
    for _, cam, img, acc in views:
        want, st, _, _ = O.render_lod(ot, cam, O.rparams(lambda_px=0.0))
        assert st == 0 and int(want.max()) > 0
        assert np.array_equal(G.u64(acc), want)
    r.close()
    t.free()
