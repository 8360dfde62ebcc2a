"""GPU parity of the 16-bit block codes (storage paragraph of the paper) against the oracle, through
the C ABI: the codes, the per-node constants and the quantised node table bit for bit; frames
drawn from the codes bit-exact against the oracle's render of its decoded tree (8-bit images
within +-1 LSB); a full-depth frame equal to the brute-force splat of the decoded points; the
batch path equal to single views; the fp32 points can be dropped."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

from gpu_helpers import NODE_FIELDS, same_floats, to_dev, u8_close

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


def _outliers_unequal(n=40000, seed=31):
    p = synth.tiny(n, seed=seed)
    xyz = p.xyz.copy()
    xyz[:4] = np.array([[1.2, 0.5, 0.5], [-0.3, 0.2, 0.1], [0.5, 1.5, 0.5], [2.0, 2.0, 2.0]], np.float32)
    mass = (p.mass * np.random.default_rng(seed).uniform(0.5, 2.0, n)).astype(np.float32)
    h = p.h.copy()
    h[10] = np.nan
    h[11] = np.inf
    return xyz, mass, h


CASES = {
    "outliers_unequal": lambda: (*_outliers_unequal(), 300),
    "tiny_equal": lambda: (*(lambda p: (p.xyz, p.mass, p.h))(synth.tiny(60000, seed=32)), 500),
    "mid_1M": lambda: (*(lambda p: (p.xyz, p.mass, p.h))(synth.mid(1 << 20, seed=33)), 16000),
}


def _both(G, xyz, mass, h, n_max, seed=5):
    t = G.build_lod(*to_dev(xyz, mass, h), n_max=n_max, seed=seed).quantize()
    ot = O.build_tree(xyz, mass, h, seed=seed, n_max=n_max)
    codes, qa, D = O.block_quantize(ot)
    return t, ot, codes, qa, D


def _compare_codes(t, codes, qa, D):
    ex = t.export_block16()
    assert np.array_equal(ex["codes"], codes), "codes differ"
    assert same_floats(ex["qa"], qa), "per-node constants differ"
    for f in NODE_FIELDS:
        a, b = ex["qnodes"][f], D.nodes[f]
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0][:5]
            raise AssertionError(f"quantised node field {f} differs at {bad}: gpu {a[bad]} oracle {b[bad]}")


@pytest.mark.parametrize("name", list(CASES))
def test_codes_and_quantised_nodes_match_oracle(G, name):
    xyz, mass, h, n_max = CASES[name]()
    t, ot, codes, qa, D = _both(G, xyz, mass, h, n_max)
    _compare_codes(t, codes, qa, D)
    assert t.info().formats == 3


def _cams():
    return {
        "outside": synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=320, height=200),
        "inside": synth.look_at((0.45, 0.55, 0.5), (0.9, 0.4, 0.6), width=333, height=197, z_near=1e-3),
        "grazing": synth.look_at((1.3, 0.5, 0.5), (0.5, 1.2, 0.4), width=160, height=120, vfov_deg=30.0),
    }


@pytest.fixture(scope="module")
def scene(G):
    xyz, mass, h = _outliers_unequal()
    return (xyz, mass, h) + _both(G, xyz, mass, h, 300)


@pytest.mark.parametrize("view", ["outside", "inside", "grazing"])
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("lam", [None, 4.0, 0.0])
def test_block16_frames_match_oracle(G, R, scene, view, kernel, lam):
    xyz, mass, h, t, ot, codes, qa, D = scene
    cam = _cams()[view]
    lam_px = G.default_lambda(300) if lam is None else lam
    img, acc = R.render(t, cam, G.make_params(lambda_px=lam_px, kernel=kernel, point_format=G.POINTS_BLOCK16))
    orp = O.rparams(lambda_px=lam_px, kernel=kernel)
    want, st, nd, npts = O.render_lod(D, cam, orp)
    assert np.array_equal(R.last_selection(), O.select(D, cam, orp))
    assert np.array_equal(G.u64(acc), want)
    assert u8_close(img.cpu().numpy(), O.tonemap(want, orp)) <= 1
    assert R.stats()["points"] == npts and R.stats()["splats"] == nd


def test_full_depth_block16_equals_bruteforce_of_decoded_points(G, R, scene):
    xyz, mass, h, t, ot, codes, qa, D = scene
    cam = _cams()["outside"]
    _, acc = R.render(t, cam, G.make_params(lambda_px=0.0, point_format=G.POINTS_BLOCK16))
    leaves = (D.nodes["flags"] & O.INTERNAL) == 0
    idx = np.concatenate([np.arange(int(x["point_first"]), int(x["point_first"]) + int(x["point_count"]))
                          for x in D.nodes[leaves]])
    P = D.pts4[idx]
    _, acc_b = R.render_bruteforce(*to_dev(np.ascontiguousarray(P[:, :3]), np.ascontiguousarray(P[:, 3]),
                                           np.ascontiguousarray(D.hs[idx])), cam, G.make_params())
    assert np.array_equal(G.u64(acc), G.u64(acc_b))


def test_tiles_and_split_frames_give_the_same_block16_image(G, R, scene):
    xyz, mass, h, t, ot, codes, qa, D = scene
    cam = _cams()["inside"]
    base = G.make_params(point_format=G.POINTS_BLOCK16, lambda_px=4.0)
    _, a0 = R.render(t, cam, base)
    ref = G.u64(a0).copy()
    for tw, th, budget in ((16, 16, 0), (64, 16, 0), (32, 32, 777)):
        _, a = R.render(t, cam, G.make_params(point_format=G.POINTS_BLOCK16, lambda_px=4.0, tile_w=tw, tile_h=th,
                                              record_budget=budget))
        assert np.array_equal(G.u64(a), ref)


def test_batch_block16_equals_single_views(G, scene):
    xyz, mass, h, t, ot, codes, qa, D = scene
    t2 = G.build_lod(*to_dev(xyz, mass, h), n_max=300, seed=9).quantize()
    rp = G.make_params(point_format=G.POINTS_BLOCK16)
    r1, rb = G.Renderer(), G.Renderer()
    cams = list(_cams().values()) + [synth.look_at((0.2, 0.9, -0.4), (0.5, 0.5, 0.5), width=96, height=64)]
    views, singles = [], []
    for k, cam in enumerate(cams):
        tree = t if k % 2 == 0 else t2
        img, acc = r1.render(tree, cam, rp)
        singles.append((img.cpu().numpy(), G.u64(acc).copy()))
        views.append((tree, cam, torch.empty_like(img), torch.empty_like(acc)))
    rb.reserve_batch(views, rp, record_capacity=1 << 24)
    rb.render_batch(views, rp)
    assert rb.status() == G.OK
    for (tree, cam, img, acc), (si, sa) in zip(views, singles):
        assert np.array_equal(G.u64(acc), sa)
        assert np.array_equal(img.cpu().numpy(), si)
    r1.close()
    rb.close()


def test_drop_float_points(G, R):
    xyz, mass, h = _outliers_unequal(20000, seed=34)
    d = to_dev(xyz, mass, h)
    t = G.build_lod(*d, n_max=300, seed=2)
    b0 = t.info().device_bytes
    cam = _cams()["outside"]
    with pytest.raises(G.GblodError) as e:
        R.render(t, cam, G.make_params(point_format=G.POINTS_BLOCK16))
    assert e.value.code == G.ERR_INVALID_ARG
    t.quantize()
    _, a = R.render(t, cam, G.make_params(point_format=G.POINTS_BLOCK16))
    ref = G.u64(a).copy()
    t.quantize(drop_float=True)
    info = t.info()
    assert info.formats == 2
    # codes (10 bytes per point) replace the fp32 points (20 bytes per point)
    assert info.device_bytes < b0
    _, a2 = R.render(t, cam, G.make_params(point_format=G.POINTS_BLOCK16))
    assert np.array_equal(G.u64(a2), ref)
    with pytest.raises(G.GblodError) as e:
        R.render(t, cam, G.make_params())
    assert e.value.code == G.ERR_INVALID_ARG
    with pytest.raises(G.GblodError):
        t.export()
    t.quantize()  # already coded: no-op


def test_block16_degenerate_trees(G, R):
    cam = _cams()["outside"]
    rp = G.make_params(point_format=G.POINTS_BLOCK16)
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    e1 = torch.zeros(0, dtype=torch.float32, device="cuda")
    t0 = G.build_lod(empty, e1, e1, n_max=10).quantize()
    _, acc = R.render(t0, cam, rp)
    assert int(G.u64(acc).sum()) == 0
    one = np.array([[0.5, 0.5, 0.5]], np.float32)
    m1, h1 = np.array([1.0], np.float32), np.array([0.01], np.float32)
    t1 = G.build_lod(*to_dev(one, m1, h1), n_max=10).quantize()
    ot = O.build_tree(one, m1, h1, seed=1, n_max=10)
    codes, qa, D = O.block_quantize(ot)
    _compare_codes(t1, codes, qa, D)
    _, acc = R.render(t1, cam, rp)
    want, _, _, _ = O.render_lod(D, cam, O.rparams(lambda_px=G.default_lambda(10)))
    assert np.array_equal(G.u64(acc), want) and want.sum() > 0
    # coincident points (a lossy leaf at depth 21)
    same = np.repeat(one, 50, axis=0)
    t2 = G.build_lod(*to_dev(same, np.ones(50, np.float32), np.full(50, 0.01, np.float32)), n_max=8).quantize()
    ot2 = O.build_tree(same, np.ones(50, np.float32), np.full(50, 0.01, np.float32), seed=1, n_max=8)
    c2, q2, D2 = O.block_quantize(ot2)
    _compare_codes(t2, c2, q2, D2)


def test_mid_workload_full_size_block16_frame(G, R):
    """Full 2^24-particle mid workload: every code and quantised node, and one 1920x1080 frame."""
    p = synth.mid()
    t = G.build_lod(*to_dev(p.xyz, p.mass, p.h), n_max=16000, seed=1).quantize()
    ot = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=16000)
    codes, qa, D = O.block_quantize(ot)
    del ot
    _compare_codes(t, codes, qa, D)
    lam = G.default_lambda(16000)
    cam = synth.helix_view(0)
    img, acc = R.render(t, cam, G.make_params(lambda_px=lam, point_format=G.POINTS_BLOCK16))
    orp = O.rparams(lambda_px=lam)
    want, st, nd, npts = O.render_lod(D, cam, orp)
    assert np.array_equal(G.u64(acc), want)
    assert u8_close(img.cpu().numpy(), O.tonemap(want, orp)) <= 1
